#!/usr/bin/env python3
"""Benchmark of the particle advance on one B300 (or N independent replicas).

Headline workload: 3D periodic 128^3 grid, turbulent B (64 Kolmogorov modes,
dB/B0 = 1), E = -v x B (solenoidal v, rms 0.01 c), 8 particles per cell
(16,777,216), relativistic Boris push with TSC gather and the deterministic
TSC deposit of the force density, FP64.  One step = part_sort + part_gather_push
(fused deposit) + part_deposit.  Metric: particle-steps/s.

Also reported on the same line: the Lagrangian-particle workload (128^3 fluid
snapshot, 4M LPs x 128 bins, RK2 or RK3 + spectral update; FP64, and with the
paired-f32 push and the deferred spectra), the 160^3 shock configuration, the
mixed form at 128^3 and 256^3, mixed-form test particles with fused steps
(2M on a 256^3 snapshot, as serving runs them), the 2D uniform-field workload
(64^2, 65,536 particles, 100 fused steps), compaction, the serving stream, the FP64 roofline
of the dominant kernel, end-to-end throughput through host buffers, and the
oracle timed on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank advances its own particles against the replicated
fields, and the ranks' deposits are summed every step (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2602_23434_b300 import synth  # noqa: E402

METRIC = ("particle-steps/s and % HBM roofline, FP64 vs mixed FP32 at stated error; "
          "serving p50/p99")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# B300 dense FP64 (non-tensor), nominal figure of the profiling notes; 2 FP64
# FMA lanes per SM-cycle on 148 SMs at the 2032 MHz maximum clock would give
# 2 x 2 x 148 x 2.032e9 = 1.20 TFLOP/s.  Reported beside the measured peak,
# which is the roofline's denominator.
FP64_NOMINAL_TFLOPS = 1.25
FALLBACK_HBM_GBS = 6400.0

# Algorithmic FP64 flops of one fused particle step (TSC, 3D, deposit on),
# FMA = 2 flops: cell coordinates 12, weights 24, gather 27*(2 mul) + 27*6*2
# = 360 (with the 9 wz*wy products counted in the 36 products), Boris 58,
# gamma + drift 17, force + deposit 7 + 9 + 27*3*2 = 178.
FLOP_PER_PSTEP_BORIS_DEP = 12 + 24 + 360 + 58 + 17 + 178
# Algorithmic HBM bytes of one particle step: state x,u read+write 96, w read 8,
# field stencil 6*8 B per cell / 8 particles per cell = 6, deposit 3*8 / 8 = 3.
BYTES_PER_PSTEP_BORIS_DEP = 96 + 8 + 6 + 3
# DRAM bytes (read + write) per particle of one launch of the FP64 brick kernel,
# from an ncu capture of the kernel on the 64^3 case of the same workload (
# 315.4 MB for 2,097,152 particles), scaled to a launch by the particle count.
TRAFFIC_PER_PARTICLE_BRICK_F64 = 315.386624e6 / 2097152  # ncu dram r+w, 64^3 capture
# FP64 arithmetic the FP64 brick kernel executes per particle-step, from the
# same capture's per-thread instruction counts (sass op dfma / dmul / dadd
# over the 2,097,152 particles): the x-quadratic gather executes fewer
# products than the method's count above, the Horner weights and the
# rsqrt / reciprocal refinements more.
FP64_OPS_PER_PSTEP_BRICK = {"dfma": 299, "dmul": 37, "dadd": 31}
# Same for the mixed brick kernel, from an ncu capture of the 128^3 case
# (1709.8 MB for 16,777,216 particles).
TRAFFIC_PER_PARTICLE_BRICK_MIXED = 1709.779712e6 / 16777216   # ncu dram r+w, 128^3 capture


# Nominal HBM3e bandwidth of a B300 (GB/s): fractions against it are reported
# beside the ones against the measured copy bandwidth.
HBM_NOMINAL_GBS = 7700.0


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- workloads
def dt_turbulent(f6, n: int, qm: float = 1.0):
    bmax = float(np.sqrt((f6[3:] ** 2).sum(axis=0)).max())
    return min(0.1 / (qm * bmax), 0.5 * (2.0 / n))


class BorisWorkload:
    """Headline FP64 workload: 128^3 turbulent, 8 ppc, Boris + TSC + deposit."""

    def __init__(self, torch, P, n=128, ppc=8, seed=1236, pseed=None):
        self.torch, self.P = torch, P
        self.n = n
        self.N = n ** 3 * ppc
        self.seed = seed
        pseed = seed if pseed is None else pseed   # particle draws (per replica)
        f = synth.em_fields(3, n, seed)
        self.dt = dt_turbulent(f, n)
        self.qm = 1.0
        dev = torch.device("cuda", torch.cuda.current_device())
        self.f = torch.as_tensor(f.reshape(6, -1)).to(dev)
        self.part = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.BORIS, capacity=self.N)
        self.part.set_fields(self.f)
        self.x = torch.empty((3, self.N), dtype=torch.float64, device=dev)
        self.u = torch.empty_like(self.x)
        self.w = torch.empty(self.N, dtype=torch.float64, device=dev)
        self.ids = torch.empty(self.N, dtype=torch.int64, device=dev)
        self.out = torch.empty((3, n ** 3), dtype=torch.float64, device=dev)
        self.part.bind(self.N, self.x, u=self.u, w=self.w, ids=self.ids)
        self.part.init_particles(pseed, 0.1)
        self.part.enable_deposit(True)
        self.part.sync()

    def step(self, ev=None):
        p = self.part
        p.sort()
        if ev is not None:
            ev[0].record(p.stream)
        p.gather_push(self.qm, self.dt, 1)
        if ev is not None:
            ev[1].record(p.stream)
        p.deposit(self.out)


def time_steps(torch, stream, fn, K: int, W: int, per_step_events=False):
    for _ in range(W):
        fn(None)
    torch.cuda.synchronize()
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)] if per_step_events else [None] * K
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(K):
        fn(kev[k])
    e1.record(stream)
    torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    kern_ms = [a.elapsed_time(b) for a, b in kev] if per_step_events else []
    return total_ms, kern_ms


# algorithmic bytes of one LP-step, the state it must read and write: the
# spectra (chi, eps: 2 x 2 x 8 B per bin), positions (2 x 24 B) and n_old
# (2 x 8 B).  The samples handed from the push to the spectral update and the
# v, B cache are the implementation's own traffic and are not counted.
def lp_step_bytes(nb):
    return 2 * 2 * 8 * nb + 48 + 16


def run_lp(torch, P, K: int, W: int, n=128, nlp=1 << 22, nb=128, seed=1238, order=2,
           fp64_tflops=None, paired=False, lazy=False):
    """The LP step of config 4: part_gather_push + spec_update, each timed.
    lazy: the deferred spectra (per-LP maps; the bins brought up to date by
    the flush that ends the timed run, which is inside the timed region)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    vel, rho, B = synth.fluid_snapshot(3, n, seed)
    f7 = torch.as_tensor(np.concatenate([vel, rho, B]).reshape(7, -1)).to(dev)
    p = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.LP_RK2, capacity=nlp, nbins=nb)
    p.set_fields(f7)
    x = torch.empty((3, nlp), dtype=torch.float64, device=dev)
    chi = torch.empty((nb, nlp), dtype=torch.float64, device=dev)
    eng = torch.empty_like(chi)
    nold = torch.empty(nlp, dtype=torch.float64, device=dev)
    p.bind(nlp, x, chi=chi, eng=eng, n_old=nold)
    p.set_lp_order(order)
    p.set_lp_arith(paired)
    p.set_spec_lazy(lazy)
    p.init_particles(seed, 0.0, 1.0, 1e6, 2.2, 1e-6)
    p.sort()                                   # once: locality of the field gathers
    p.sync()
    dt = 0.5 * 2.0 / n
    # cooling break near eps ~ 1e3 after 100 steps with <U_B> = (B0^2 + dB^2)/2 = 1
    c0 = 1.0 / (1e3 * 1.0 * 100 * dt)
    calls = [0]
    push_ev = []              # (start, end) of each timed step's push

    def step(ev):
        if ev is not None:
            e = torch.cuda.Event(enable_timing=True)
            e.record(p.stream)
            push_ev.append(e)
        p.gather_push(0.0, dt, 1)
        if ev is not None:
            ev[0].record(p.stream)
        p.spec_update(dt, c0, 0.0)
        if ev is not None:
            ev[1].record(p.stream)
        calls[0] += 1
        if calls[0] == W + K:  # spectra back as (chi, eps), inside the timed region
            p.flush()

    l0 = p.launches()
    kev = []
    total, kern = time_steps(torch, p.stream, lambda ev: (kev.append(ev), step(ev)), K, W,
                             per_step_events=True)
    p.sync()
    launches = (p.launches() - l0) // (K + W)
    ms = total / K
    spec_ms = float(np.mean(kern))
    kev = [e for e in kev if e is not None]
    spec_bytes = nlp * 2 * 2 * nb * 8
    hbm, hbm_kind = peaks()
    arith = ("push in paired-f32 arithmetic (~48-bit), FP64 state and spectra" if paired
             else "FP64")
    if lazy:
        arith += (f"; spectra deferred as per-LP maps, brought up to date once per {K} steps "
                  f"(the flush ending the timed run)")
    # deferred spectra: per step the state and the per-LP map (3 doubles read
    # and written); the bins once per timed run (the flush that ends it)
    step_bytes = (48 + 16 + 48 + 2 * 2 * 8 * nb / K) if lazy else lp_step_bytes(nb)
    step_hbm = {"bytes_per_lp_step": step_bytes,
                "achieved_GBps": step_bytes * nlp / (total / K / 1e3) / 1e9,
                "frac": step_bytes * nlp / (total / K / 1e3) / 1e9 / hbm,
                "frac_of_nominal": step_bytes * nlp / (total / K / 1e3) / 1e9 / HBM_NOMINAL_GBS,
                "peak_kind": hbm_kind}
    if lazy:
        step_hbm["what"] = (f"positions, n_old and the per-LP map every step, the spectra once "
                            f"per {K} steps; the eager update moves {lp_step_bytes(nb)} B per "
                            f"LP-step")
    push_ms = float(np.mean([a.elapsed_time(e[0]) for a, e in zip(push_ev, kev)]))
    # the two bounds of the step: the push on the FP64 pipe (FP64 instructions
    # per LP-step with the TSC x quadratics: 425 for RK2 by an ncu count, 513
    # for RK3 = that plus the third stencil's 120 of the weight form less its 32
    # saved; at 2 per SM-cycle = half the measured FP64 FLOP/s), the spectral
    # update on HBM
    slots = 425 if order == 2 else 513
    del chi, eng
    if paired:
        push_roof = {"bound": "f32 issue (paired-f32 arithmetic)", "kernel_ms": push_ms,
                     "fp64_kernel_bound_ms_at_measured_peak": (
                         nlp * slots / (fp64_tflops * 1e12 / 2) * 1e3 if fp64_tflops else None)}
    else:
        push_roof = {"bound": "fp64 pipe", "slots_per_lp_step": slots,
                     "bound_ms_at_measured_peak": (
                         nlp * slots / (fp64_tflops * 1e12 / 2) * 1e3
                         if fp64_tflops else None),
                     "frac": (nlp * slots / (fp64_tflops * 1e12 / 2) * 1e3 / push_ms
                              if fp64_tflops else None),
                     "kernel_ms": push_ms}
    return {"workload": f"LP 3D {n}^3 snapshot, {nlp} LPs x {nb} bins, "
                        f"{'RK2' if order == 2 else 'SSP-RK3'} + TSC + spectra, {arith}",
            "value": nlp * K / (total / 1e3), "unit": "LP-steps/s", "ms_per_step": ms,
            "spec_update_ms": spec_ms,
            "spec_update_GBps": spec_bytes / (spec_ms / 1e3) / 1e9,
            "push_ms": push_ms,
            "step_hbm": step_hbm,
            "roofline_step": {
                "push": push_roof,
                "spec_update": {"bound": "hbm", "bytes": spec_bytes,
                                "bound_ms": spec_bytes / (hbm * 1e9) * 1e3,
                                "kernel_ms": spec_ms,
                                "frac": spec_bytes / (spec_ms / 1e3) / 1e9 / hbm,
                                "frac_of_nominal":
                                    spec_bytes / (spec_ms / 1e3) / 1e9 / HBM_NOMINAL_GBS}},
            "c0": c0, "dt": dt, "gpu_launches_per_step": launches}


def run_compact(torch, P, n=128, ppc=8, fracs=(0.01, 0.1), K=10, seed=1240):
    """Sec. 3.2 hole/filler compaction of the headline FP64 state (x, u, w, id:
    64 B per particle) with a random fraction of the particles flagged.  Each
    timed call starts from the same restored state (the restore is untimed).
    Algorithmic bytes: the mask (1 B per particle), each filler's record read
    and written (2 x 64 B), and the rows after the first of x and u moved to
    the new row stride (2 x 4 x 8 B per survivor)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    N = n ** 3 * ppc
    p = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.BORIS, capacity=N)
    x = torch.empty((3, N), dtype=torch.float64, device=dev)
    u, w = torch.empty_like(x), torch.empty(N, dtype=torch.float64, device=dev)
    ids = torch.empty(N, dtype=torch.int64, device=dev)
    p.bind(N, x, u=u, w=w, ids=ids)
    p.init_particles(seed, 0.1)
    p.sync()
    keep = [t.clone() for t in (x, u, w, ids)]
    hbm, hbm_kind = peaks()
    out = {"workload": f"{N} FP64 particles (128^3 x 8), x, u, w, id; random deletion",
           "unit": "GB/s", "peak": hbm, "peak_kind": hbm_kind, "cases": []}
    rng = np.random.default_rng(seed)
    for frac in fracs:
        d = rng.random(N) < frac
        nk = int(N - d.sum())
        nfill = int(d[:nk].sum())
        dmask = torch.as_tensor(d.astype(np.uint8)).to(dev)
        ms = []
        for k in range(K + 3):
            for t, s0 in zip((x, u, w, ids), keep):
                t.copy_(s0)
            p.bind(N, x, u=u, w=w, ids=ids)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(p.stream)
            got = p.compact(dmask)
            e1.record(p.stream)
            torch.cuda.synchronize()
            assert got == nk
            if k >= 3:
                ms.append(e0.elapsed_time(e1))
        t = float(np.median(ms))
        alg = N + 2 * 64 * nfill + 2 * 4 * 8 * nk
        out["cases"].append({"deleted_frac": frac, "n_new": nk, "fillers": nfill, "ms": t,
                             "particles_per_s": N / (t / 1e3),
                             "algorithmic_bytes": alg, "achieved_GBps": alg / (t / 1e3) / 1e9,
                             "frac": alg / (t / 1e3) / 1e9 / hbm,
                             "frac_of_nominal": alg / (t / 1e3) / 1e9 / HBM_NOMINAL_GBS})
    del keep, x, u, w, ids
    return out


def run_lp_shock(torch, P, K: int, W: int, n=160, ppc=4, nb=128, seed=1241, paired=False,
                 lazy=False):
    """The paper's shock configuration per GPU (Sec. 4.1.2 extended to 3D,
    Sec. 5): a stationary planar shock at x = 0 (Rankine-Hugoniot, rho_u = 50,
    v_u = 0.1, r = 40/11, B = (1, 0, 0)) on a 160^3 grid, 4 LPs per cell
    (16.4M), each with 128 bins on [1e2, 1e4], p = 9; step = Heun RK2 + TSC
    gather, smooth spectral update, shock detection and Eq.
    convolution_spectra for the LPs entering the shock.  paired / lazy: the
    paired-f32 push and the deferred spectra (brought up to date by the flush
    that ends the timed run)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    r = 40.0 / 11.0
    xc = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    down = np.broadcast_to(xc > 0.0, (n, n, n))
    f7 = np.zeros((7, n, n, n))
    f7[0] = np.where(down, 0.1 / r, 0.1)
    f7[3] = np.where(down, 50.0 * r, 50.0)
    f7[4] = 1.0
    N = n ** 3 * ppc
    p = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.LP_RK2, capacity=N, nbins=nb)
    p.set_fields(torch.as_tensor(f7.reshape(7, -1)).to(dev))
    del f7
    x = torch.empty((3, N), dtype=torch.float64, device=dev)
    chi = torch.empty((nb, N), dtype=torch.float64, device=dev)
    eng = torch.empty_like(chi)
    nold = torch.empty(N, dtype=torch.float64, device=dev)
    st = torch.zeros(N, dtype=torch.uint8, device=dev)
    p.bind(N, x, chi=chi, eng=eng, n_old=nold)
    p.set_lp_arith(paired)
    p.set_spec_lazy(lazy)
    p.init_particles(seed, 0.0, 1e2, 1e4, 9.0, 1e-6)
    p.sort()
    p.enable_shocks(1.5, st)
    p.sync()
    dt = 0.5 * (2.0 / n) / 0.1

    calls = [0]

    def step(ev):
        p.gather_push(0.0, dt, 1)
        if ev is not None:
            ev[0].record(p.stream)
        p.spec_update(dt, 1e-8, 0.0)
        if ev is not None:
            ev[1].record(p.stream)
        calls[0] += 1
        if calls[0] == W + K:  # spectra back as (chi, eps), inside the timed region
            p.flush()

    l0 = p.launches()
    total, kern = time_steps(torch, p.stream, step, K, W, per_step_events=True)
    p.sync()
    launches = (p.launches() - l0) // (K + W)
    in_shock = int(st.sum().item())
    ms = total / K
    spec_ms = float(np.mean(kern))
    del chi, eng
    arith = "paired-f32 push (~48-bit), FP64 state and spectra" if paired else "FP64"
    if lazy:
        arith += f"; spectra deferred, brought up to date once per {K} steps"
    return {"workload": f"LP 3D stationary planar shock (Rankine-Hugoniot, r = 40/11) {n}^3, "
                        f"{N} LPs x {nb} bins on [1e2, 1e4], p = 9, RK2 + TSC + spectra + "
                        f"shock detection + Eq. convolution_spectra, {arith}",
            "value": N * K / (total / 1e3), "unit": "LP-steps/s", "ms_per_step": ms,
            "spec_update_and_shock_ms": spec_ms, "lps_in_shock_cells_at_end": in_shock,
            "paper_context": "Particles_RK#1 + RK#2 + Spectra = 341 ms per step for 1.65e7 "
                             "LPs on one A100 of a Leonardo node (paper's timing table)",
            "dt": dt, "gpu_launches_per_step": launches}


# Mixed form: per particle-step, state read 44 B (cell 4, offsets 12, the
# momentum as a compensated f32 pair 24, w 4) + written 40 B, f32 field
# stencil 6 x 4 B per cell / 8 ppc = 3, deposit partials 3 x 8 B per cell /
# 8 ppc = 3.
BYTES_PER_PSTEP_MIXED_DEP = 44 + 40 + 3 + 3


class MixedWorkload:
    """Mixed form: int32 cell + f32 offsets, the momentum as a compensated f32
    pair, f32 push and fields; deposit sums in f32 within a source cell's
    particles, two-float across cells, FP64 across bricks; turbulent fields;
    Boris + TSC + deposit."""

    def __init__(self, torch, P, n, ppc, seed, with_ids=False):
        dev = torch.device("cuda", torch.cuda.current_device())
        self.n, self.N = n, n ** 3 * ppc
        f = synth.em_fields(3, n, seed)
        self.dt = dt_turbulent(f, n)
        self.f = torch.as_tensor(f.reshape(6, -1).astype(np.float32)).to(dev)
        del f
        self.part = P.Part(P.make_grid(3, n), P.MIXED, P.TSC, P.BORIS, capacity=self.N)
        self.part.set_fields(self.f)
        self.cell = torch.empty(self.N, dtype=torch.int32, device=dev)
        self.off = torch.empty((3, self.N), dtype=torch.float32, device=dev)
        self.u = torch.empty((6, self.N), dtype=torch.float32, device=dev)  # (hi, lo) pair
        self.w = torch.empty(self.N, dtype=torch.float32, device=dev)
        self.ids = torch.empty(self.N, dtype=torch.int64, device=dev) if with_ids else None
        self.out = torch.empty((3, n ** 3), dtype=torch.float64, device=dev)
        self.part.bind(self.N, self.cell, off=self.off, u=self.u, w=self.w, ids=self.ids)
        self.part.init_particles(seed, 0.1)
        self.part.enable_deposit(True)
        self.part.sync()

    def step(self, ev=None):
        p = self.part
        p.sort()
        if ev is not None:
            ev[0].record(p.stream)
        p.gather_push(1.0, self.dt, 1)
        if ev is not None:
            ev[1].record(p.stream)
        p.deposit(self.out)


def run_mixed(torch, P, n, ppc, K, W, seed):
    wl = MixedWorkload(torch, P, n, ppc, seed)
    l0 = wl.part.launches()
    total, kern = time_steps(torch, wl.part.stream, wl.step, K, W, per_step_events=True)
    wl.part.sync()
    km = float(np.mean(kern))
    hbm, kind = peaks()
    gbs = BYTES_PER_PSTEP_MIXED_DEP * wl.N / (km / 1e3) / 1e9
    res = {"workload": f"3D {n}^3 turbulent, {wl.N} particles ({ppc}/cell), mixed form "
                       "(int32 cell + f32 offset, u as a compensated f32 pair, f32 push/fields; "
                       "deposit: f32 sums within a source cell, two-float across cells, FP64 "
                       "across bricks), "
                       "Boris + TSC + deposit",
           "value": wl.N * K / (total / 1e3), "unit": "particle-steps/s",
           "ms_per_step": total / K, "push_kernel_ms": km,
           "roofline_push": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                             "frac": gbs / hbm, "peak_kind": kind,
                             "frac_of_nominal": gbs / HBM_NOMINAL_GBS,
                             "bytes_per_particle_step": BYTES_PER_PSTEP_MIXED_DEP,
                             "traffic": TRAFFIC_PER_PARTICLE_BRICK_MIXED * wl.N},
           "gpu_launches_per_step": (wl.part.launches() - l0) // (K + W)}
    del wl
    torch.cuda.empty_cache()
    return res


def mixed_error_vs_fp64(torch, P, n=128, ppc=8, steps=20, seed=1236):
    """Same seed, same fields: FP64 and mixed runs of `steps` steps, matched by
    particle id; max position difference (cells) and momentum error."""
    m = MixedWorkload(torch, P, n, ppc, seed, with_ids=True)
    d = BorisWorkload(torch, P, n, ppc, seed)
    for _ in range(steps):
        m.step()
        d.step()
    m.part.sync()
    d.part.sync()
    im = torch.argsort(m.ids)
    idd = torch.argsort(d.ids)
    dx = 2.0 / n
    c = m.cell[im].to(torch.int64)
    j = torch.stack([c % n, (c // n) % n, c // (n * n)]).to(torch.float64)
    xm = -1.0 + (j + 0.5 + m.off[:, im].to(torch.float64)) * dx
    xd = d.x[:, idd]
    dd = (xm - xd) / dx
    dd = dd - n * torch.round(dd / n)
    um = m.u[:3, im].to(torch.float64) + m.u[3:, im].to(torch.float64)
    ud = d.u[:, idd]
    du = (um - ud).norm(dim=0) / ud.norm(dim=0)
    gm = torch.sqrt(1 + (um * um).sum(0))
    gd = torch.sqrt(1 + (ud * ud).sum(0))
    res = {"steps": steps, "particles": m.N,
           "max_position_error_cells": float(dd.abs().max()),
           "median_position_error_cells": float(dd.abs().median()),
           "max_rel_momentum_error": float(du.max()),
           "median_rel_momentum_error": float(du.median()),
           "max_energy_error": float((gm / gd - 1).abs().max()),
           "deposit_rel_l2_error": float((m.out - d.out).norm() / d.out.norm())}
    del m, d
    torch.cuda.empty_cache()
    return res


def run_serving(torch, requests=200, seed=1239, load=0.7, budget_gb=16.0, round_ms=10.0):
    """Poisson stream of test-particle requests against 4 resident snapshots
    (128^3 x2, 256^3 x2, turbulent, f32): N log-uniform in [1e3, 1e7],
    steps log-uniform in [10, 1000], mixed precision, admitted by device
    memory, batched by the persistent graph-replayed kernel.  The arrival rate
    is `load` x the autotuned capacity / E[N steps]."""
    from paper_2602_23434_b300 import serving as S
    cap = 10 ** 7
    snaps = [S.make_snapshot(torch, 128, seed, cap), S.make_snapshot(torch, 128, seed + 1, cap),
             S.make_snapshot(torch, 256, seed + 2, cap), S.make_snapshot(torch, 256, seed + 3, cap)]
    tune = S.autotune(torch, snaps, n=1 << 22,
                      cache_path=os.path.join(ROOT, "_build", "autotune.json"))
    rate = tune["psteps_per_s"]
    en = (1e7 - 1e3) / np.log(1e4)
    es = (1000 - 10) / np.log(100)
    lam = load * rate / (en * es)
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / lam, requests)
    arrivals = np.cumsum(gaps)
    ns = np.exp(rng.uniform(np.log(1e3), np.log(1e7), requests)).astype(np.int64)
    steps = np.exp(rng.uniform(np.log(10), np.log(1000), requests)).astype(np.int64)
    which = rng.integers(0, 4, requests)
    srv = S.Server(torch, snaps, int(budget_gb * 2 ** 30), chunk=tune["chunk"],
                   slice_steps=tune["slice_steps"], threads=tune["threads"],
                   ctas_per_sm=tune["ctas_per_sm"], keep_results=False,
                   round_psteps=rate * round_ms / 1e3 if round_ms else None)
    t0 = time.perf_counter()
    srv.clock = lambda: time.perf_counter() - t0
    k = 0
    while k < requests or srv.queue or srv.active or srv.inflight:
        now = srv.clock()
        while k < requests and arrivals[k] <= now:
            srv.submit(int(which[k]), int(ns[k]), int(steps[k]), seed=seed * 1000 + k,
                       arrival=float(arrivals[k]))
            k += 1
        if not srv.round():
            # nothing to enqueue: poll again shortly (rounds in flight, or the
            # next arrival), so arrivals are admitted while the GPU works
            nxt = arrivals[k] - srv.clock() if k < requests else 0.001
            time.sleep(max(0.0, min(0.0005, nxt)))
    srv.drain()
    wall = srv.clock()
    st = srv.stats()
    srv.close()
    res = {"workload": f"{requests} Poisson requests at {load:.0%} of measured capacity, "
                       "N ~ logU[1e3, 1e7], steps ~ logU[10, 1000], 4 resident snapshots "
                       "(128^3 x2, 256^3 x2, f32), mixed precision",
           "value": st["particle_steps"] / wall, "unit": "particle-steps/s",
           "throughput_busy": st["throughput_busy"], "p50_s": st["p50_s"],
           "p99_s": st["p99_s"], "rounds": st["rounds"], "wall_s": wall,
           "arrival_rate_per_s": lam, "capacity_psteps_per_s": rate,
           "autotune": {k2: tune[k2] for k2 in ("threads", "ctas_per_sm", "chunk",
                                                 "slice_steps")},
           "pipeline": "two work lists: round k + 1 staged and enqueued while round k runs; "
                       "admission (device init + sort) enqueued without host synchronisation",
           "round_budget": f"{round_ms} ms of capacity per round, shared equally by the "
                           f"active requests (whole remainders that fit are done at once)"}
    del snaps
    torch.cuda.empty_cache()
    return res


def run_mixed_fused(torch, P, n=256, N=1 << 21, steps=16, reps=5, seed=1239):
    """Test particles in the mixed form, as serving runs them: N sorted
    particles on an n^3 turbulent snapshot (sparser than one per cell at the
    defaults), `steps` fused steps per call (part_gather_push), no deposit."""
    dev = torch.device("cuda", torch.cuda.current_device())
    f = torch.as_tensor(synth.em_fields(3, n, seed).reshape(6, -1).astype(np.float32)).to(dev)
    p = P.Part(P.make_grid(3, n), P.MIXED, P.TSC, P.BORIS, capacity=N)
    p.set_fields(f)
    cell = torch.empty(N, dtype=torch.int32, device=dev)
    off = torch.empty((3, N), dtype=torch.float32, device=dev)
    u = torch.empty((6, N), dtype=torch.float32, device=dev)
    p.bind(N, cell, off=off, u=u)
    p.init_particles(7, 0.1)
    p.sort()
    p.flush()
    p.sync()
    dt = 0.5 * 2.0 / n

    def run(ev):
        p.gather_push(1.0, dt, steps)

    total, _ = time_steps(torch, p.stream, run, reps, 3)
    p.sync()
    return {"workload": f"mixed form, {N} sorted test particles on a {n}^3 turbulent snapshot, "
                        f"{steps} fused Boris steps per call (k_boris_particles_mixed)",
            "value": N * steps * reps / (total / 1e3), "unit": "particle-steps/s",
            "ms_per_call": total / reps}


def run_2d(torch, P, n=64, ppc=16, steps=100, seed=1235):
    dev = torch.device("cuda", torch.cuda.current_device())
    N = n * n * ppc
    f = torch.as_tensor(synth.uniform_em_fields(2, n, B=(0, 0, 1.0)).reshape(6, -1)).to(dev)
    p = P.Part(P.make_grid(2, n), P.FP64, P.TSC, P.BORIS, capacity=N)
    p.set_fields(f)
    x = torch.empty((3, N), dtype=torch.float64, device=dev)
    u = torch.empty_like(x)
    p.bind(N, x, u=u)
    p.init_particles(seed, 0.1)
    p.sort()
    p.sync()
    dt = 0.1

    def run(ev):
        p.gather_push(1.0, dt, steps)

    total, _ = time_steps(torch, p.stream, run, 5, 3)
    p.sync()
    return {"workload": f"2D {n}^2 uniform B, {N} particles, {steps} fused Boris steps, FP64",
            "value": N * steps * 5 / (total / 1e3), "unit": "particle-steps/s",
            "ms_per_run": total / 5}


def fp64_peak_measured(torch, P, stream):
    """The FP64 FMA rate of this GPU, measured now (part_probe_fp64_fma: 16
    independent DFMA chains per thread, 4 CTAs of 256 threads per SM, best of
    5 launches), with the SM clock read just after."""
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    tf, ms = P.probe_fp64_fma(stream.cuda_stream, sink, ctas_per_sm=4, iters=8192, reps=5)
    sm = None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()),
                              "--query-gpu=clocks.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=10).stdout.strip()
        sm = float(out.splitlines()[0])
    except Exception:
        pass
    return tf, {"tflops": tf, "best_launch_ms": ms, "sm_mhz_after": sm,
                "what": "independent DFMA chains on every SM, CUDA events, best of 5"}


# ----------------------------------------------------------------------------- e2e
def run_e2e(torch, wl: BorisWorkload, K: int):
    """The step as a coupled code runs it through the C ABI: the particles stay
    resident on the device (the state the library advances), while every step
    the host supplies the fields (E, B from the fluid solver: H2D from pinned
    memory, padded by part_set_fields) and reads back the deposited force
    density (D2H).  Copies run on a second stream, double-buffered, so the H2D
    of step k+1 and the D2H of step k overlap the computation; every step's
    bytes cross the bus inside the timed region.  Two more figures: the same
    step with the pinned host buffers handed to the C ABI directly (the
    kernels read and write them over the host link), and one that also moves
    the whole particle state both ways every step, serialised."""
    N = wl.N
    s = wl.part.stream
    cs = torch.cuda.Stream()
    hf = [torch.empty(wl.f.shape, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    for h in hf:
        h.copy_(wl.f)
    df = [torch.empty_like(wl.f) for _ in range(2)]
    hout = [torch.empty(wl.out.shape, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    dout = [torch.empty_like(wl.out) for _ in range(2)]
    hx = torch.empty((3, N), dtype=torch.float64, pin_memory=True)
    hu = torch.empty_like(hx, pin_memory=True)
    hw = torch.empty(N, dtype=torch.float64, pin_memory=True)
    wl.part.sync()
    hx.copy_(wl.x)
    hu.copy_(wl.u)
    hw.copy_(wl.w)
    ev = lambda: torch.cuda.Event()  # noqa: E731

    def fields_run(K):
        h2d_done = [ev(), ev()]
        padded = [ev(), ev()]
        dep_done = [ev(), ev()]
        d2h_done = [ev(), ev()]
        with torch.cuda.stream(cs):
            df[0].copy_(hf[0], non_blocking=True)
            h2d_done[0].record(cs)
        for k in range(K):
            b = k & 1
            if k + 1 < K:  # fields of the next step, once their buffer is free
                with torch.cuda.stream(cs):
                    if k >= 1:
                        cs.wait_event(padded[1 - b])
                    df[1 - b].copy_(hf[1 - b], non_blocking=True)
                    h2d_done[1 - b].record(cs)
            s.wait_event(h2d_done[b])
            if k >= 2:
                s.wait_event(d2h_done[b])          # dout[b] read back by then
            wl.part.set_fields(df[b])
            padded[b].record(s)
            p = wl.part
            p.sort()
            p.gather_push(wl.qm, wl.dt, 1)
            p.deposit(dout[b])
            dep_done[b].record(s)
            with torch.cuda.stream(cs):
                cs.wait_event(dep_done[b])
                hout[b].copy_(dout[b], non_blocking=True)
                d2h_done[b].record(cs)
        torch.cuda.synchronize()

    def state_step():
        with torch.cuda.stream(s):
            wl.x.copy_(hx, non_blocking=True)
            wl.u.copy_(hu, non_blocking=True)
            wl.w.copy_(hw, non_blocking=True)
            wl.f.copy_(hf[0], non_blocking=True)
            wl.part.set_fields(wl.f)
            wl.step()
            wl.part.flush()
            hx.copy_(wl.x, non_blocking=True)
            hu.copy_(wl.u, non_blocking=True)
            hout[0].copy_(wl.out, non_blocking=True)
        s.synchronize()

    def host_buffers_run(K):
        # the C ABI given host buffers directly: the padding kernel reads the
        # pinned snapshot and the combine kernel writes the pinned deposit
        p = wl.part
        for _ in range(K):
            p.set_fields(hf[0])
            p.sort()
            p.gather_push(wl.qm, wl.dt, 1)
            p.deposit(hout[0])
        torch.cuda.synchronize()

    fields_run(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fields_run(K)
    r_fields = N * K / (time.perf_counter() - t0)
    host_buffers_run(2)
    t0 = time.perf_counter()
    host_buffers_run(K)
    r_host = N * K / (time.perf_counter() - t0)
    wl.part.set_fields(wl.f)
    state_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        state_step()
    torch.cuda.synchronize()
    r_state = N * K / (time.perf_counter() - t0)
    f_b = hf[0].numel() * 8
    o_b = hout[0].numel() * 8
    st_b = (hx.numel() + hu.numel()) * 8
    return {"value": r_fields, "unit": "particle-steps/s", "h2d_bytes_per_step": f_b,
            "d2h_bytes_per_step": o_b,
            "what": "particles resident; per step H2D of the field snapshot (E, B) and D2H "
                    "of the deposited force density, overlapped with the computation",
            "c_abi_host_buffers": {"value": r_host, "unit": "particle-steps/s",
                                   "h2d_bytes_per_step": f_b, "d2h_bytes_per_step": o_b,
                                   "what": "pinned host field snapshot passed to part_set_fields "
                                           "and pinned host output to part_deposit: the kernels "
                                           "read and write them over the host link, no copies"},
            "state_roundtrip": {"value": r_state, "unit": "particle-steps/s",
                                "h2d_bytes_per_step": f_b + st_b + hw.numel() * 8,
                                "d2h_bytes_per_step": o_b + st_b}}


# ----------------------------------------------------------------------------- oracle
def executed_fp64(N, kernel_ms, peak_tflops):
    """The FP64 arithmetic the brick kernel executes (ncu counts per
    particle-step), as a rate against the measured FP64 peak."""
    ops = FP64_OPS_PER_PSTEP_BRICK
    flop = 2 * ops["dfma"] + ops["dmul"] + ops["dadd"]
    tf = flop * N / (kernel_ms / 1e3) / 1e12
    return {"fp64_ops_per_particle_step": dict(ops), "flop_per_particle_step": flop,
            "achieved": tf, "frac": tf / peak_tflops if peak_tflops else None,
            "source": "ncu sass thread-instruction counts of the 64^3 capture"}


def headline_config(grid: int, particles: int, dt: float, world: int) -> dict:
    """The `config` object of the headline line (both arms)."""
    return {"workload": "3D periodic 128^3, B = z + turbulent dB (64 Kolmogorov modes, "
                        "dB/B0 = 1), E = -v x B (solenoidal v, rms 0.01 c), "
                        "16,777,216 particles (8/cell), u_th = 0.1, step = sort + "
                        "Boris/TSC gather + TSC force deposit, FP64",
            "particles": particles, "grid": [grid] * 3, "dt": dt,
            "l2": "inputs larger than L2 (about 2 GB of state, fields and deposit "
                  "touched per step vs 126 MB L2); no flush",
            "parallelism": ("one GPU" if world == 1 else
                            f"{world} ranks: particles partitioned (each rank its own "
                            f"16,777,216), fields replicated, deposit summed across ranks "
                            f"every step in rank order")}


def _oracle_boris_stepper(n: int, seed: int, deposit: bool = True):
    """(one_step, grid, dt) of the oracle on the turbulent n^3 workload: keys,
    stable sort, permute, Boris step, deposit (or the Boris step alone for
    test particles)."""
    from oracle import oracle as O
    f = synth.em_fields(3, n, seed).reshape(6, -1)
    g = O.make_grid(3, (n, n, n))
    dt = dt_turbulent(f.reshape(6, n, n, n), n)
    brick = (8, 8, 8)

    def one_step(x, u, w):
        if not deposit:
            x1, u1, _, _ = O.boris_step(g, O.TSC, f, x, u, w, 1.0, dt, False)
            return x1, u1, w
        k = O.keys(g, brick, x)
        perm = O.stable_sort(k)
        x, u, w = x[:, perm], u[:, perm], w[perm]
        x1, u1, F, xo = O.boris_step(g, O.TSC, f, x, u, w, 1.0, dt, True)
        O.deposit(g, O.TSC, xo, F)
        return x1, u1, w

    return one_step, g, dt


def _sample_size(one_step, init, budget_s: float, steps: int, n_max: int) -> int:
    """Particles per sampled step so that `steps` steps take about budget_s."""
    ns = 1 << 16
    x, u, w = init(ns)
    t0 = time.perf_counter()
    one_step(x, u, w)
    t1 = max(time.perf_counter() - t0, 1e-3)
    return int(min(n_max, max(1 << 14, ns * budget_s / steps / t1)))


def cpu_baseline(budget_s: float = 15.0, n=128, seed=1236):
    """The oracle as it stands (OpenMP over particles in the push; sort and
    deposit sequential), one step = keys + stable sort + permute + Boris step
    + deposit, on a sample of the headline workload's particles."""
    from oracle import oracle as O
    one_step, g, dt = _oracle_boris_stepper(n, seed)

    def init(k):
        x, u, w, _ = O.init_particles(g, k, seed, 0.1)
        return x, u, w

    # one host thread first, on a small sample
    cores = O.max_threads()
    O.set_threads(1)
    N1 = 1 << 16
    x, u, w = init(N1)
    t0 = time.perf_counter()
    one_step(x, u, w)
    e1 = time.perf_counter() - t0
    O.set_threads(cores)
    steps = 3
    Ns = _sample_size(one_step, init, budget_s, steps, 1 << 23)
    x, u, w = init(Ns)
    t0 = time.perf_counter()
    for _ in range(steps):
        x, u, w = one_step(x, u, w)
    el = time.perf_counter() - t0
    return {"value": Ns * steps / el, "unit": "particle-steps/s", "cores": cores,
            "kind": "oracle", "dt": dt,
            "single_thread": {"value": N1 / e1, "unit": "particle-steps/s",
                              "sample": f"{N1} particles, 1 step"},
            "sample": f"{Ns} of the 16,777,216 particles of the 128^3 workload, {steps} "
                      f"steps (keys, stable sort, permute, Boris step, deposit), {el:.1f} s"}


def cpu_baseline_mixed(budget_s: float = 8.0, n=256, seed=1237):
    """The oracle (FP64: it has no mixed form) on the mixed-form workload's
    inputs: the turbulent 256^3 fields, a sample of its 134,217,728
    particles, sort + Boris + deposit, in the same unit."""
    from oracle import oracle as O
    one_step, g, _ = _oracle_boris_stepper(n, seed)

    def init(k):
        x, u, w, _ = O.init_particles(g, k, seed, 0.1)
        return x, u, w

    steps = 2
    Ns = _sample_size(one_step, init, budget_s, steps, 1 << 22)
    x, u, w = init(Ns)
    t0 = time.perf_counter()
    for _ in range(steps):
        x, u, w = one_step(x, u, w)
    el = time.perf_counter() - t0
    return {"value": Ns * steps / el, "unit": "particle-steps/s", "cores": O.max_threads(),
            "kind": "oracle",
            "sample": f"{Ns} of the 134,217,728 particles of the 256^3 mixed-form workload, "
                      f"{steps} steps of the FP64 oracle (keys, stable sort, permute, Boris "
                      f"step, deposit), {el:.1f} s"}


def cpu_baseline_lp(budget_s: float = 8.0, n=128, nb=128, seed=1238):
    """The oracle on the LP workload: the 128^3 fluid snapshot, a sample of
    its 4,194,304 LPs with 128 bins each, Heun RK2 + spectral update."""
    from oracle import oracle as O
    vel, rho, B = synth.fluid_snapshot(3, n, seed)
    vel, rho, B = vel.reshape(3, -1), rho.reshape(1, -1), B.reshape(3, -1)
    g = O.make_grid(3, (n, n, n))
    dt = 0.5 * 2.0 / n
    c0 = 1.0 / (1e3 * 1.0 * 100 * dt)
    e0, x0 = O.init_spectrum(nb, 1.0, 1e6, 2.2, 1e-6)

    def init(k):
        x = np.random.default_rng(seed).uniform(-1.0, 1.0, (3, k))
        chi = np.repeat(x0[:, None], k, axis=1)
        eng = np.repeat(e0[:, None], k, axis=1)
        _, n_new, _, _ = O.lp_rk2_step(g, O.TSC, vel, rho, B, x, 0.0)
        return x, (chi, eng), n_new

    def one_step(x, spec, n_old):
        x, n_new, b2m, gam = O.lp_rk2_step(g, O.TSC, vel, rho, B, x, dt)
        chi, eng, n_old = O.spec_update(spec[0], spec[1], n_old, n_new, b2m, gam, dt, c0)
        return x, (chi, eng), n_old

    steps = 2
    Ns = _sample_size(one_step, init, budget_s, steps, 1 << 20)
    x, spec, n_old = init(Ns)
    t0 = time.perf_counter()
    for _ in range(steps):
        x, spec, n_old = one_step(x, spec, n_old)
    el = time.perf_counter() - t0
    return {"value": Ns * steps / el, "unit": "LP-steps/s", "cores": O.max_threads(),
            "kind": "oracle",
            "sample": f"{Ns} of the 4,194,304 LPs x {nb} bins of the 128^3 LP workload, "
                      f"{steps} steps (Heun RK2 + spectral update), {el:.1f} s"}


def cpu_baseline_serving(budget_s: float = 6.0, n=256, seed=1241):
    """No-batching reference for the serving stream: the oracle advances
    one request's test particles alone (FP64 Boris steps, no deposit) on a
    256^3 snapshot; a request of N particles and S steps would take N S /
    rate seconds on the host cores."""
    from oracle import oracle as O
    one_step, g, _ = _oracle_boris_stepper(n, seed, deposit=False)

    def init(k):
        x, u, w, _ = O.init_particles(g, k, seed, 0.1)
        return x, u, w

    steps = 3
    Ns = _sample_size(one_step, init, budget_s, steps, 1 << 22)
    x, u, w = init(Ns)
    t0 = time.perf_counter()
    for _ in range(steps):
        x, u, w = one_step(x, u, w)
    el = time.perf_counter() - t0
    rate = Ns * steps / el
    med = np.exp(0.5 * (np.log(1e3) + np.log(1e7))) * np.exp(0.5 * (np.log(10) + np.log(1000)))
    return {"value": rate, "unit": "particle-steps/s", "cores": O.max_threads(),
            "kind": "oracle",
            "sample": f"one request of {Ns} test particles on a 256^3 snapshot, {steps} FP64 "
                      f"Boris steps alone (no batching), {el:.1f} s",
            "median_request_s": med / rate,
            "largest_request_s": 1e7 * 1000 / rate}


def reference_arm(args):
    """The oracle, timed on the host cores, on the headline workload's config
    and metric: W untimed and K timed steps, each step one pass of keys,
    stable sort, permute, Boris step and deposit over a bounded sample of the
    16,777,216 particles, sized so that the run ends within about two
    minutes.  value = sampled particles x K / timed seconds."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    n, seed = 128, 1236
    one_step, g, dt = _oracle_boris_stepper(n, seed)

    def init(k):
        x, u, w, _ = O.init_particles(g, k, seed, 0.1)
        return x, u, w

    K, W = args.steps, args.warmup
    Ns = _sample_size(one_step, init, 90.0, K + W, 128 ** 3 * 8)
    x, u, w = init(Ns)
    for _ in range(W):
        x, u, w = one_step(x, u, w)
    t0 = time.perf_counter()
    for _ in range(K):
        x, u, w = one_step(x, u, w)
    el = time.perf_counter() - t0
    value = Ns * K / el
    N = 128 ** 3 * 8
    sample = (f"{Ns} of the {N} particles of the 128^3 workload per step, {W} warm-up + {K} "
              f"timed steps (keys, stable sort, permute, Boris step, deposit), {el:.1f} s timed")
    cfg = headline_config(128, N, dt, 1)
    cfg["parallelism"] = f"the oracle, OpenMP over particles on {O.max_threads()} host cores"
    cfg["sample_particles_per_step"] = Ns
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": K, "warmup": W, "ms_per_step": el / K * 1e3,
            "higher_is_better": True, "scaling": "weak", "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": "particle-steps/s",
                             "cores": O.max_threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- main
def only(args):
    """One secondary workload at --grid cells per axis (profiling captures)."""
    import torch
    from paper_2602_23434_b300 import _lib as P
    from paper_2602_23434_b300.build import build
    build()
    if args.only == "mixed":
        res = run_mixed(torch, P, args.grid, 8, args.steps, args.warmup, 1237)
    elif args.only in ("shock", "shock_paired_lazy"):
        res = run_lp_shock(torch, P, max(3, args.steps), 3, n=args.grid,
                           paired=args.only != "shock", lazy=args.only != "shock")
    elif args.only == "compact":
        res = run_compact(torch, P, n=args.grid, K=max(3, args.steps))
    elif args.only in ("lp", "lp_paired", "lp_lazy", "lp_paired_lazy"):
        res = run_lp(torch, P, args.steps, args.warmup, n=args.grid,
                     nlp=max(1 << 16, 2 * args.grid ** 3), paired="paired" in args.only,
                     lazy=args.only.endswith("lazy"))
    elif args.only == "mixed_fused":
        res = run_mixed_fused(torch, P, n=args.grid, reps=max(1, args.steps))
    elif args.only == "boris2d":
        res = run_2d(torch, P)
    else:
        res = run_serving(torch, requests=args.serve_requests)
    print(json.dumps({"only": args.only, "grid": args.grid, **res}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-extras", action="store_true", help="headline workload only")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests in the serving stream (the stated stream is 2000)")
    ap.add_argument("--grid", type=int, default=128,
                    help="cells per axis of the headline workload (128 = the stated one; "
                         "smaller only for profiling captures)")
    ap.add_argument("--only", choices=["mixed", "lp", "lp_paired", "lp_lazy", "lp_paired_lazy",
                                       "serving", "compact", "shock", "shock_paired_lazy",
                                       "boris2d", "mixed_fused"],
                    default=None,
                    help="run one secondary workload alone at --grid cells per axis and print "
                         "its result (for profiling captures); no headline line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    if args.only:
        return only(args)

    import torch
    from paper_2602_23434_b300 import _lib as P
    from paper_2602_23434_b300.build import build

    from paper_2602_23434_b300 import replicas as R
    rank, world, local = R.env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        build()
    if dist:
        dist.barrier()

    wl = BorisWorkload(torch, P, n=args.grid, seed=1236, pseed=R.rank_seed(1236, rank))
    stream = wl.part.stream
    l0 = wl.part.launches()
    step = wl.step
    if world > 1:
        # particles partitioned over the ranks (each its own set), fields
        # replicated: every step the ranks' deposits are summed in rank order
        # (all-to-all of slices, part_sum_ordered, all-gather) so every rank
        # holds the whole deposit, the same bits on every rank
        from paper_2602_23434_b300 import multirank as M
        ops = M.LibOps(wl.part, wl.N)

        def step(ev=None):
            wl.step(ev)
            wl.out.view(-1).copy_(M.combine_replicated(ops, dist, wl.out.view(-1)))
    # warm-up
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    l1 = wl.part.launches()
    total_ms, kern_ms = time_steps(torch, stream, step, args.steps, 0, per_step_events=True)
    launches = wl.part.launches() - l1
    clocks = clk.stop()
    wl.part.sync()
    total_ms = R.max_over_ranks(total_ms, dist, device="cuda")
    value = R.job_rate(wl.N, args.steps, world, total_ms / 1e3)
    kmean = float(np.mean(kern_ms))
    hbm, hbm_kind = peaks()
    achieved_tf = FLOP_PER_PSTEP_BORIS_DEP * wl.N / (kmean / 1e3) / 1e12
    achieved_gbs = BYTES_PER_PSTEP_BORIS_DEP * wl.N / (kmean / 1e3) / 1e9
    fp64_peak, fp64_probe = fp64_peak_measured(torch, P, stream)

    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": headline_config(args.grid, wl.N, wl.dt, world),
        "roofline": {"bound": "alu", "kernel": "k_boris_brick_f64_dep (TSC, 3D, warp-specialised push + deposit)",
                     "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved_tf / fp64_peak, "peak_kind": "measured",
                     "peak_probe": fp64_probe,
                     "peak_nominal": FP64_NOMINAL_TFLOPS,
                     "frac_of_nominal": achieved_tf / FP64_NOMINAL_TFLOPS,
                     "traffic": TRAFFIC_PER_PARTICLE_BRICK_F64 * wl.N,
                     "traffic_unit": "bytes per launch (ncu dram read+write, scaled by "
                                     "particles from the 64^3 capture)",
                     "flop_per_particle_step": FLOP_PER_PSTEP_BORIS_DEP,
                     "executed": executed_fp64(wl.N, kmean, fp64_peak),
                     "kernel_ms": kmean,
                     "peak_note": "FP64 non-tensor FMA rate measured on this GPU by "
                                  "part_probe_fp64_fma right after the timed steps (burst); "
                                  "peak_nominal is the recipe's nominal figure"},
        "roofline_hbm": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                         "frac": achieved_gbs / hbm,
                         "frac_of_nominal": achieved_gbs / HBM_NOMINAL_GBS,
                         "bytes_per_particle_step": BYTES_PER_PSTEP_BORIS_DEP,
                         "peak_kind": hbm_kind},
        "clocks": clocks, "gpu_launches": launches,
    }
    if rank == 0:
        line["e2e"] = run_e2e(torch, wl, max(3, args.steps // 4))
    del wl
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_extras:
        try:
            line["lp"] = run_lp(torch, P, max(5, args.steps // 2), 3, fp64_tflops=fp64_peak)
        except Exception as e:  # report, do not hide
            line["lp"] = {"error": repr(e)}
        try:
            line["lp_rk3"] = run_lp(torch, P, max(5, args.steps // 2), 3, order=3,
                                    fp64_tflops=fp64_peak)
        except Exception as e:
            line["lp_rk3"] = {"error": repr(e)}
        for key, order, paired, lazy in (("lp_paired", 2, True, False),
                                         ("lp_rk3_paired", 3, True, False),
                                         ("lp_lazy", 2, False, True),
                                         ("lp_paired_lazy", 2, True, True)):
            try:
                line[key] = run_lp(torch, P, max(5, args.steps // 2), 3, order=order,
                                   fp64_tflops=fp64_peak, paired=paired, lazy=lazy)
            except Exception as e:
                line[key] = {"error": repr(e)}
        try:
            line["boris_2d"] = run_2d(torch, P)
        except Exception as e:
            line["boris_2d"] = {"error": repr(e)}
        try:
            line["mixed_fused"] = run_mixed_fused(torch, P)
        except Exception as e:
            line["mixed_fused"] = {"error": repr(e)}
        try:
            mx = run_mixed(torch, P, 128, 8, args.steps, 3, 1236)
            mx["speedup_vs_fp64_same_workload"] = mx["value"] / value
            line["mixed_128"] = mx
            line["mixed_256"] = run_mixed(torch, P, 256, 8, max(5, args.steps // 2), 3, 1237)
            line["mixed_error_vs_fp64"] = mixed_error_vs_fp64(torch, P)
            # the stated case: 256^3, 134M particles, 200 steps
            line["mixed_error_vs_fp64_256"] = mixed_error_vs_fp64(torch, P, n=256, steps=200,
                                                                  seed=1237)
        except Exception as e:
            line["mixed"] = {"error": repr(e)}
        try:
            line["lp_shock"] = run_lp_shock(torch, P, max(5, args.steps // 2), 3)
        except Exception as e:
            line["lp_shock"] = {"error": repr(e)}
        try:
            line["lp_shock_paired_lazy"] = run_lp_shock(torch, P, max(5, args.steps // 2), 3,
                                                        paired=True, lazy=True)
        except Exception as e:
            line["lp_shock_paired_lazy"] = {"error": repr(e)}
        try:
            line["compact"] = run_compact(torch, P)
        except Exception as e:
            line["compact"] = {"error": repr(e)}
        try:
            line["serving"] = run_serving(torch, requests=args.serve_requests)
        except Exception as e:
            line["serving"] = {"error": repr(e)}
    if rank == 0 and not args.no_cpu:
        cb = cpu_baseline()
        cb.pop("dt", None)
        line["cpu_baseline"] = cb
        if not args.no_extras:
            rows = {}
            for key, fn in (("lp", cpu_baseline_lp), ("mixed_256", cpu_baseline_mixed),
                            ("serving", cpu_baseline_serving)):
                try:
                    rows[key] = fn()
                except Exception as e:  # report, do not hide
                    rows[key] = {"error": repr(e)}
            line["cpu_baseline_rows"] = rows
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
