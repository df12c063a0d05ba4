#!/usr/bin/env python
"""Throughput of the Vicsek step on GB300: particle-updates/s at N = 2^24.

Workload: standard Vicsek model, N = 2^24 = 16,777,216 particles, L = 2896
(rho = 2.0004), R = 1, v0 = 0.5, eta = 0.45, periodic, uniform isotropic random
initial state (seeded Philox), one step = collision + streaming for every
particle with p(t) measured on the fly.  The state (268 MB per buffer) is
larger than L2, so no flush is needed between steps.

Prints one JSON line.  --impl reference times the FP64 oracle instead, on the
host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_FULL = 1 << 24
L_FULL = 2896.0
ALG_BYTES = 32          # per particle-update: 16 B record read + 16 B written
METRIC = "particle-updates/s (N*steps/s) at N=2^24, rho=2"
UNIT = "particle-updates/s"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in self.lines:
            if not (t0 <= ts <= t1):
                continue
            f = [s.strip() for s in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


class NvmlClockSampler:
    """SM clock and clock-event reasons read through NVML (the driver's
    libnvidia-ml, by ctypes) every couple of milliseconds, so that a timed
    region of a few tens of milliseconds still gets a dozen samples.  Reads
    only; changes no setting.  start() returns False when NVML is not there
    (the caller then falls back to the nvidia-smi sampler)."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, uuid: str | None, index: int, period_s: float = 0.002):
        self.uuid, self.index, self.period = uuid, index, period_s
        self.lines = []
        self.stop_flag = threading.Event()
        self.t = None

    def start(self) -> bool:
        import ctypes as C

        try:
            nv = C.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return False
            dev = C.c_void_p()
            rc = 1
            if self.uuid:
                u = self.uuid if self.uuid.startswith("GPU-") else "GPU-" + self.uuid
                rc = nv.nvmlDeviceGetHandleByUUID(u.encode(), C.byref(dev))
            if rc != 0:
                rc = nv.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.index), C.byref(dev))
            if rc != 0:
                return False
            mx = C.c_uint(0)
            nv.nvmlDeviceGetMaxClockInfo(dev, 1, C.byref(mx))          # NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
            get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
        except (OSError, AttributeError):
            return False
        self.nv, self.dev, self.get_reasons = nv, dev, get_reasons

        def run():
            clk, rs = C.c_uint(0), C.c_ulonglong(0)
            while not self.stop_flag.is_set():
                if self.nv.nvmlDeviceGetClockInfo(self.dev, 1, C.byref(clk)) == 0 and \
                        self.get_reasons(self.dev, C.byref(rs)) == 0:
                    self.lines.append((time.perf_counter(), float(clk.value), int(rs.value)))
                time.sleep(self.period)

        self.t = threading.Thread(target=run, daemon=True)
        self.t.start()
        return True

    def stop(self):
        self.stop_flag.set()
        if self.t:
            self.t.join(timeout=5)

    def summary(self, t0, t1):
        sm, reasons = [], set()
        for ts, mhz, bits in self.lines:
            if t0 <= ts <= t1:
                sm.append(mhz)
                for b, name in self.REASONS.items():
                    if bits & b:
                        reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvml"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for fn in ("aap_kernels.cu", "aap_pipe.cu", "aap_tile.cuh", "aap_internal.cuh", "aap_device.cuh"):
        with open(os.path.join(ROOT, "paper_2211_15630_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(n):
    """DRAM bytes per k_step launch from the committed ncu summary, or None
    when the kernel source changed since the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_step_traffic.json")) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_hash") != _kernel_hash():
        return None
    return float(d["bytes_per_particle"]) * n


def replica_throughput(ms_local, units_per_rank, world, dist=None, device="cpu"):
    """Whole-job throughput of `world` independent replicas (one per rank, no
    data-path collective): the units all ranks processed over the slowest
    rank's time (a MAX all-reduce of the per-rank milliseconds).  Returns
    (units per second, max ms)."""
    import torch

    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return world * units_per_rank / (ms_max / 1e3), ms_max


def _cpu_baseline(eta, budget_s=20.0):
    """The oracle as it stands, on all host cores, on the full workload for as
    many steps as fit in about budget_s seconds (at least one)."""
    import oracle as O

    O.build()
    cores = os.cpu_count() or 1
    m = O.Model(n=N_FULL, lx=L_FULL, ly=L_FULL, r=1.0, v=0.5, eta=eta, seed=1)
    x, y, th = O.init_state(m)
    steps, t_used = 0, 0.0
    while t_used < budget_s and steps < 50:
        t0 = time.perf_counter()
        x, y, th, _ = O.run(m, x, y, th, steps, 1, threads=cores)
        t_used += time.perf_counter() - t0
        steps += 1
    return {"value": N_FULL * steps / t_used, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} full steps of the N=2^24, L=2896 workload from the Philox initial "
                      f"state ({t_used:.1f} s, OpenMP over {cores} threads)"}


def _structure_factor(rho_counts):
    """Radially averaged S(k) = <|rho_hat(k)|^2> / N of a density-count field."""
    import numpy as np

    n = rho_counts.sum()
    d = rho_counts - rho_counts.mean()
    f = np.abs(np.fft.fft2(d)) ** 2 / max(n, 1.0)
    ky = np.fft.fftfreq(d.shape[0]) * d.shape[0]
    kx = np.fft.fftfreq(d.shape[1]) * d.shape[1]
    kk = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
    kb = np.rint(kk).astype(int)
    kmax = min(d.shape) // 2
    s = np.array([f[kb == k].mean() for k in range(1, kmax)])
    return s


def _bench_brownian(A, W, torch, stream, steps):
    p = W.brownian_walls(seed=1)
    h = A.aap_create(p, stream.cuda_stream)
    A.aap_step(h, 20)
    A.aap_sync(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    A.aap_step(h, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    A.aap_destroy(h)
    return {"workload": "langevin_N2^20_L724_reflecting_dt0.01", "updates_per_s": p.n * steps / (ms / 1e3),
            "ms_per_step": ms / steps, "steps": steps}


def _bench_coarse(A, W, torch, stream, peak, frames=50):
    """Coarse-grained fields (density, polarisation per bin): the surrogate's
    N = 524,288, L = 512 state into 128 x 128 bins, and an N = 2^24, L = 2896
    state into 724 x 724 bins; whole calls (clear, bin, finish) timed with
    events over back-to-back frames.  Algorithmic bytes: the 16 B record of
    every particle read once (the fields themselves are small)."""
    out = {}
    for name, p, nb in (("sur_N524288_L512_128x128", W.surrogate_training(eta=0.4, seed=3), 128),
                        ("vicsek_N2^24_L2896_724x724", W.vicsek_large(seed=5), 724)):
        h = A.aap_create(p, stream.cuda_stream)
        A.aap_step(h, 20)
        f = torch.empty(3 * nb * nb, device="cuda", dtype=torch.float32)
        A.aap_coarse_grain(h, nb, nb, f.data_ptr())
        A.aap_sync(h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(frames):
            A.aap_coarse_grain(h, nb, nb, f.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / frames
        gbs = 16.0 * p.n / (us * 1e-6) / 1e9
        out[name] = {"us_per_frame": us, "particles_per_s": p.n / (us * 1e-6), "achieved_gbs": gbs,
                     "frac_of_hbm": gbs / peak}
        A.aap_destroy(h)
    return out


def _bench_metric_free(A, W, torch, stream, steps, kn=6):
    """mfVM (k nearest neighbours, Sec. 2.3) at N = 2^24, L = 2896: whole
    steps timed with events, then the kernel split from the library's timers."""
    p = W.metric_free_vicsek(kn=kn, seed=1)
    h = A.aap_create(p, stream.cuda_stream)
    A.aap_step(h, 20)
    A.aap_sync(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    A.aap_step(h, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    A.aap_set_timing(h, True)
    A.aap_step(h, 20)
    A.aap_sync(h)
    kms, kl = A.aap_get_timing(h)
    A.aap_set_timing(h, False)
    A.aap_destroy(h)
    return {"workload": f"mfvm_k{kn}_N2^24_L2896", "updates_per_s": p.n * steps / (ms / 1e3),
            "ms_per_step": ms / steps, "steps": steps,
            "search_update_kernels_ms": kms[0] / max(kl[0], 1), "finish_ms": kms[1] / max(kl[1], 1)}


def _bench_ensemble(A, W, torch, stream, steps, long_steps=5000, trial_steps=50):
    """256 Vicsek replicas (N log-uniform 2^10..2^18, rho in {0.5,1,2,4}, eta in
    [0.1,0.7]): one batched, graph-replayed launch per step vs the same replicas
    run one after another as standalone systems with the same tile shapes
    (`steps` steps each), then the configured run: `long_steps` measured steps
    of the whole ensemble and the time-averaged p of every replica."""
    import numpy as np

    ps = W.ensemble_replicas(count=256, seed=7)
    ntot = sum(p.n for p in ps)
    e = A.aap_ens_create(ps, stream.cuda_stream)
    pol, trial = A.aap_ens_autotune(e, trial_steps)
    A.aap_ens_step(e, 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    A.aap_ens_step(e, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_ens = e0.elapsed_time(e1)
    layouts = [A.aap_ens_get_layout(e, r) for r in range(len(ps))]
    ms_seq = 0.0
    exact = True
    for r, p in enumerate(ps):
        q = A.aap_params_default()
        for f, _ in A.aap_params._fields_:
            setattr(q, f, getattr(p, f))
        q.tile_w, q.tile_h, q.threads = layouts[r].tile_w, layouts[r].tile_h, layouts[r].threads
        h = A.aap_create(q, stream.cuda_stream)
        A.aap_step(h, 3)
        torch.cuda.synchronize()
        e0.record(stream)
        A.aap_step(h, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_seq += e0.elapsed_time(e1)
        if r in (0, 255):
            a = A.aap_get_state(h, q.n)
            b = A.aap_ens_get_state(e, r, q.n)
            exact = exact and all(np.array_equal(u, v) for u, v in zip(a, b))
        A.aap_destroy(h)
    # the configured run: long_steps measured steps (Sec. 3.4 window), <p> per replica
    torch.cuda.synchronize()
    e0.record(stream)
    A.aap_ens_measure(e, long_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_long = e0.elapsed_time(e1)
    pm = A.aap_ens_phi_mean(e)
    etas = np.array([p.eta for p in ps])
    A.aap_ens_destroy(e)
    return {"workload": "256 Vicsek replicas, N log-uniform [2^10,2^18], rho {0.5,1,2,4}, eta U[0.1,0.7]",
            "replicas": len(ps), "total_particles": ntot, "steps": steps,
            "updates_per_s": ntot * steps / (ms_ens / 1e3),
            "sequential_updates_per_s": ntot * steps / (ms_seq / 1e3),
            "speedup_vs_sequential": ms_seq / ms_ens, "policy": int(pol),
            "policy_trial_steps": trial_steps,
            "policy_ms_per_step": [round(float(v), 4) for v in trial],
            "phi_error": 0.0 if exact else None, "replicas_bitwise_equal_checked": [0, 255],
            "measured_steps": long_steps, "measured_updates_per_s": ntot * long_steps / (ms_long / 1e3),
            "measured_ms_per_step": ms_long / long_steps,
            "phi_mean_eta_below_0.3": [round(float(v), 4) for v in np.percentile(pm[etas < 0.3], [0, 50, 100])],
            "phi_mean_eta_above_0.5": [round(float(v), 4) for v in np.percentile(pm[etas > 0.5], [0, 50, 100])]}


def _surrogate_data(A, W, torch, stream, train_traj=200, steps=2000, every=10):
    """Training fields of the learned surrogate at its stated size: Vicsek
    N = 524,288, L = 512 trajectories (eta uniform in [0.3, 0.5], seeds
    10000 + r) from the Philox initial state, advanced together as one
    batched ensemble and coarse-grained to 128 x 128 x 3 every `every` steps
    (steps / every + 1 frames each, kept on the device: 7.9 GB at 200 x 2000)."""
    import numpy as np

    nb = 128
    g = np.random.default_rng(3)
    etas = g.uniform(0.3, 0.5, train_traj)
    ps = [W.surrogate_training(eta=float(etas[r]), seed=10000 + r) for r in range(train_traj)]
    e = A.aap_ens_create(ps, stream.cuda_stream)
    nfr = steps // every + 1
    frames = torch.zeros(train_traj, nfr, 3, nb, nb, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(nfr):
        for r in range(train_traj):
            A.aap_ens_coarse_grain(e, r, nb, nb, frames[r, k].data_ptr())
        if k + 1 < nfr:
            A.aap_ens_step(e, every)
    stream.synchronize()
    A.aap_ens_destroy(e)
    t_data = time.perf_counter() - t0
    return {"frames": frames, "etas": etas, "train_traj": train_traj, "steps": steps, "every": every,
            "nfr": nfr, "data_s": t_data,
            "particle_updates_per_s": train_traj * 524288 * steps / t_data}


def _bench_surrogate(A, W, torch, stream, data, iters=3000, horizon=100, lr=2e-3, pushforward=0.0, conserve=0):
    """Train the field surrogate on `data` (_surrogate_data), then advance
    held-out states by `horizon` particle steps with the surrogate and with
    the particle method; report speedup and the errors in p and S(k), beside
    those of keeping the fields unchanged."""
    import numpy as np

    nb, every = 128, data["every"]
    g = np.random.default_rng(3)
    frames, etas, train_traj, nfr = data["frames"], data["etas"], data["train_traj"], data["nfr"]
    t_data = data["data_s"]
    B = 32
    s = A.aap_sur_create(A.aap_sur_params_default(nbx=nb, nby=nb, max_batch=B, lr=lr, seed=11, conserve=conserve),
                         stream.cuda_stream)
    xin = torch.zeros(B, 3, nb, nb, device="cuda")
    xtg = torch.zeros_like(xin)
    eta_t = torch.zeros(B, device="cuda")
    etas_t = torch.tensor(etas, dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    loss = 0.0
    npf = int(round(pushforward * B))
    for it in range(iters):
        # pushforward: part of the batch starts from the network's own
        # one-application prediction (no gradient through it) and targets the
        # frame two applications ahead, which keeps long rollouts stable
        pf = npf if it >= iters // 4 else 0
        ri = torch.from_numpy(g.integers(0, train_traj, B)).cuda()
        ki = torch.from_numpy(g.integers(0, nfr - 2, B)).cuda()
        xin.copy_(frames[ri, ki])
        eta_t.copy_(etas_t[ri])
        if pf:
            A.aap_sur_predict(s, xin.data_ptr(), eta_t.data_ptr(), pf, 1, xin.data_ptr())
            xtg[:pf].copy_(frames[ri[:pf], ki[:pf] + 2])
        xtg[pf:].copy_(frames[ri[pf:], ki[pf:] + 1])
        loss = A.aap_sur_train_step(s, xin.data_ptr(), xtg.data_ptr(), eta_t.data_ptr(), B)
    t_train = time.perf_counter() - t0
    # held-out evaluation
    errs, keep_errs, sk_errs, sk_keep, t_part, t_sur = [], [], [], [], 0.0, 0.0
    apps = horizon // every
    f0 = torch.zeros(1, 3, nb, nb, device="cuda")
    ft = torch.zeros_like(f0)
    fp = torch.zeros_like(f0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    area = (512.0 / nb) ** 2
    held_out = np.linspace(0.3, 0.5, 16)          # 16 held-out seeds 20000..20015 over the eta range
    ed = torch.zeros(1, device="cuda")
    # the first call captures the predict graph for these buffers; later calls replay it
    A.aap_sur_predict(s, f0.data_ptr(), ed.data_ptr(), 1, apps, fp.data_ptr())
    torch.cuda.synchronize()
    starts = (300, 1500)                              # both inside the time range of the training frames
    for j, eta in enumerate(held_out):
        p = W.surrogate_training(eta=float(eta), seed=20000 + j)
        h = A.aap_create(p, stream.cuda_stream)
        done = 0
        for t_start in starts:
            A.aap_step(h, t_start - done)
            A.aap_coarse_grain(h, nb, nb, f0.data_ptr())
            torch.cuda.synchronize()
            ev0.record(stream)
            A.aap_step(h, horizon)
            A.aap_coarse_grain(h, nb, nb, ft.data_ptr())
            ev1.record(stream)
            torch.cuda.synchronize()
            done = t_start + horizon
            t_part += ev0.elapsed_time(ev1)
            ed.fill_(float(eta))
            ev0.record(stream)
            A.aap_sur_predict(s, f0.data_ptr(), ed.data_ptr(), 1, apps, fp.data_ptr())
            ev1.record(stream)
            torch.cuda.synchronize()
            t_sur += ev0.elapsed_time(ev1)
            a_t, a_p, a_0 = (v.cpu().numpy()[0].astype(np.float64) for v in (ft, fp, f0))
            phi = lambda f: np.hypot(f[1].sum(), f[2].sum()) / f[0].sum()
            errs.append(abs(phi(a_p) - phi(a_t)))
            keep_errs.append(abs(phi(a_0) - phi(a_t)))
            s_t, s_p, s_0 = (_structure_factor(f[0] * area) for f in (a_t, a_p, a_0))
            sk_errs.append(float(np.linalg.norm(s_p - s_t) / np.linalg.norm(s_t)))
            sk_keep.append(float(np.linalg.norm(s_0 - s_t) / np.linalg.norm(s_t)))
        A.aap_destroy(h)
    A.aap_sur_destroy(s)
    nev = len(errs)
    return {"workload": "Vicsek N=524288 L=512 eta[0.3,0.5] -> 128x128x3 fields, 4-layer 3x3 conv 32 ch",
            "train_trajectories": train_traj, "steps_per_trajectory": data["steps"],
            "frames_per_trajectory": nfr, "iterations": iters,
            "data_particle_updates_per_s": data["particle_updates_per_s"],
            "batch": B, "lr": lr, "pushforward": pushforward, "conserve": conserve, "final_loss": loss, "data_s": t_data, "train_s": t_train,
            "horizon_steps": horizon, "speedup_vs_particles": t_part / t_sur,
            "particle_ms": t_part / nev, "surrogate_ms": t_sur / nev,
            "held_out_states": nev, "held_out_seeds": len(held_out), "start_steps": list(starts),
            "phi_abs_error": float(np.mean(errs)), "phi_abs_error_keep_fields": float(np.mean(keep_errs)),
            "sk_rel_l2_error": float(np.mean(sk_errs)), "sk_rel_l2_error_keep_fields": float(np.mean(sk_keep))}


def run_reference(args, rank, world):
    """--impl reference: the oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return 0
    import oracle as O

    O.build()
    cores = os.cpu_count() or 1
    n_s, l_s = 1 << 16, 181.0           # same density (rho = 2.0003), same per-particle work
    m = O.Model(n=n_s, lx=l_s, ly=l_s, r=1.0, v=0.5, eta=args.eta, seed=1)
    x, y, th = O.init_state(m)
    x, y, th, _ = O.run(m, x, y, th, 0, args.warmup, threads=cores)
    t0 = time.perf_counter()
    x, y, th, _ = O.run(m, x, y, th, args.warmup, args.steps, threads=cores)
    dt = time.perf_counter() - t0
    val = n_s * args.steps / dt
    sample = (f"each step a full update of a 2^16-particle sample of the workload at the same "
              f"density (L=181, rho=2.0003, eta={args.eta}); {args.steps} steps in {dt:.2f} s")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "vicsek_N2^24_L2896_rho2", "sample_n": n_s, "eta": args.eta},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--eta", type=float, default=0.45)
    ap.add_argument("--n", type=int, default=N_FULL)
    ap.add_argument("--L", type=float, default=L_FULL)
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--clock-window", type=float, default=1.0,
                    help="seconds of steps under the clock sampler, the timed ones included")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--tile", type=str, default="0x0")
    ap.add_argument("--kn", type=int, default=0,
                    help="k > 0: the metric-free variant (k nearest neighbours, Sec. 2.3) of the workload")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    import paper_2211_15630_gb300 as A
    from paper_2211_15630_gb300 import build as B

    if rank == 0 or world == 1:
        B.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        B.build()
    stream = torch.cuda.Stream()
    tw, th_ = (int(v) for v in args.tile.split("x"))

    def make(eta, seed):
        p = A.aap_params_default(n=args.n, lx=args.L, ly=args.L, r=1.0, v=0.5, eta=eta,
                                 seed=seed, threads=args.threads, tile_w=tw, tile_h=th_, kn=args.kn)
        return p, A.aap_create(p, stream.cuda_stream)

    def timed(h, k):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        A.aap_step(h, k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    p, h = make(args.eta, 1 + rank)
    lay = A.aap_get_layout(h)
    tw0 = time.perf_counter()
    A.aap_step(h, args.warmup)
    A.aap_sync(h)
    est_s = max((time.perf_counter() - tw0) / max(args.warmup, 1), 1e-5)
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except (AttributeError, RuntimeError):
        uuid = None
    clocks = NvmlClockSampler(uuid, local)
    if not clocks.start():
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
    # clock window: the same steps run for at least a second under the
    # sampler, then the state and step counter are put back (the noise is
    # counter based, so the timed steps are exactly those a run without the
    # window would take); the window's samples include the timed region's
    t_window = time.perf_counter()
    soak = int(math.ceil(args.clock_window / est_s)) - args.steps
    if soak > 0:
        snap = A.aap_get_state(h, args.n)
        step0 = A.aap_observe(h).step
        A.aap_step(h, soak)
        A.aap_sync(h)
        A.aap_set_state(h, *snap, step=step0)
        del snap
        torch.cuda.synchronize()
    A.aap_set_timing(h, True)
    t_begin = time.perf_counter()
    ms = timed(h, args.steps)
    t_end = time.perf_counter()
    kms, klaunch = A.aap_get_timing(h)
    A.aap_set_timing(h, False)
    clocks.stop()
    A.aap_sync(h)
    obs = A.aap_observe(h)
    value, ms_max = replica_throughput(ms, args.n * args.steps, world, dist, "cuda")

    # end to end through the C ABI with host buffers: upload the state from
    # pinned memory, K steps recording p(t) into host memory, download the state
    xs, ys, ts = A.aap_get_state(h, args.n)
    px = torch.from_numpy(xs).pin_memory().numpy()
    py = torch.from_numpy(ys).pin_memory().numpy()
    pt = torch.from_numpy(ts).pin_memory().numpy()
    # page-locked host buffers for the state read back at the end
    ox = torch.empty(args.n, dtype=torch.float64).pin_memory().numpy()
    oy = torch.empty(args.n, dtype=torch.float64).pin_memory().numpy()
    ot = torch.empty(args.n, dtype=torch.float32).pin_memory().numpy()
    ke = args.e2e_steps
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    A.aap_set_state(h, px, py, pt, step=obs.step)
    phi = A.aap_phi_trace(h, ke)
    xs2, ys2, ts2 = A.aap_get_state(h, args.n, out=(ox, oy, ot))
    e2e_s = time.perf_counter() - t0
    e2e_val, _ = replica_throughput(e2e_s * 1e3, args.n * ke, world, dist, "cuda")
    state_bytes = args.n * (8 + 8 + 4)
    A.aap_destroy(h)

    extras = {}
    if not args.no_extras and world == 1:
        from paper_2211_15630_gb300 import workloads as W

        for eta in (0.2, 0.7):
            if abs(eta - args.eta) < 1e-9:
                continue
            pe, he = make(eta, 1)
            A.aap_step(he, args.warmup)
            msx = timed(he, max(args.steps // 4, 50))
            extras[f"vicsek_eta_{eta}_updates_per_s"] = args.n * max(args.steps // 4, 50) / (msx / 1e3)
            A.aap_destroy(he)
        extras["brownian"] = _bench_brownian(A, W, torch, stream, 10000)
        extras["metric_free"] = _bench_metric_free(A, W, torch, stream, 100)
        extras["ensemble"] = _bench_ensemble(A, W, torch, stream, 200)
        extras["coarse_grain"] = _bench_coarse(A, W, torch, stream, _peaks()[0])
        with torch.cuda.stream(stream):     # torch copies and library calls share one stream
            # conserving (grid means of density and polarisation kept) and free
            data = _surrogate_data(A, W, torch, stream)
            extras["surrogate"] = _bench_surrogate(A, W, torch, stream, data, conserve=3)
            extras["surrogate_unconstrained"] = _bench_surrogate(A, W, torch, stream, data, conserve=0)
            del data

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    peak, peak_kind = _peaks()
    kstep_ms = kms[0] / max(klaunch[0], 1)
    achieved = ALG_BYTES * args.n / (kstep_ms / 1e3) / 1e9
    traffic = _traffic(args.n) if args.kn == 0 else None
    csum = clocks.summary(t_window, t_end)
    csum["window_s"] = round(t_end - t_window, 3)
    csum["window_steps"] = max(soak, 0) + args.steps
    csum["samples_timed_region"] = clocks.summary(t_begin, t_end)["samples"]
    default_size = args.n == N_FULL and args.L == L_FULL
    workload = ("vicsek_N2^24_L2896_rho2" if default_size else f"vicsek_N{args.n}_L{args.L:g}")
    if args.kn:
        workload = "mf" + workload + f"_k{args.kn}"
    step_kernel = ("k_step_pipe" if lay.threads == 1024 else "k_step") if args.kn == 0 else \
        "k_mf_count+scan+scatter+update+exact"
    launches_per_step = 2 if args.kn == 0 else 7
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (uniform isotropic Philox initial state)",
        "config": {"workload": workload, "n": args.n, "L": args.L, "R": 1.0, "kn": args.kn,
                   "v0": 0.5, "eta": args.eta, "boundary": "periodic", "l2": "state > L2 (no flush)",
                   "tile": [lay.tile_w, lay.tile_h], "threads": lay.threads,
                   "stage_cap": lay.stage_cap, "parallelism": "replicas only" if world > 1 else "1 gpu"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": step_kernel,
                     "kernel_ms": kstep_ms, "peak_kind": peak_kind,
                     "alg_bytes_per_update": ALG_BYTES},
        "step_kernels_ms": {step_kernel: kstep_ms, "k_finish": kms[1] / max(klaunch[1], 1)},
        "e2e": {"value": e2e_val, "unit": UNIT, "steps": ke,
                "h2d_bytes_per_step": state_bytes / ke,
                "d2h_bytes_per_step": (state_bytes + 8 * (ke + 1)) / ke},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": csum,
        "phi_end": float(phi[-1]),
        "mean_neighbours": obs.mean_neighbours,
        "frac_of_hbm_roofline": value * ALG_BYTES / (peak * 1e9),
    }
    if extras:
        line["extras"] = extras
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(args.eta)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
