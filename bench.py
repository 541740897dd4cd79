#!/usr/bin/env python3
"""Throughput of the coupled LBM + Stokeslet-fit Langevin step on GB300.

One step = one full pass of the hot path: particle gather / Stokeslet fit /
Philox random force / Langevin update / reaction-force accumulation, VACF
accumulation (lag 5000), fused pull-stream + BGK collision over the whole
lattice, and the body-force term at the particle nodes.

Default workload: 256^3 periodic box (FP32 deviation storage), tau = 0.8,
16384 Brownian particles (M = 10, gamma = 0.5, kT = 1e-4, uniformly random
positions, Maxwellian velocities), VACF to lag 5000.  value = lattice
updates per second (MLUPS) over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lbp|reference]

Under torchrun (N > 1) every rank runs its own replica box (replicas only, no
collective in the step) and the timing is the max over ranks.
--impl reference times the FP64 CPU oracle on this host's cores instead.
"""
from __future__ import annotations

import argparse
import contextlib
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1909_13412_gb300 import workloads as wl  # noqa: E402
from paper_1909_13412_gb300.lbp import AUTOTUNE_SHAPES  # noqa: E402  (names only; loads no library)

METRIC = "MLUPS and % HBM roofline per GB300 at fixed accuracy vs FP64 oracle; plain vs BF16/batched"
# algorithmic bytes per node update: 15 loads + 15 stores of the stored deviation
BYTES_PER_NODE = {"f32": 2 * 15 * 4, "bf16": 2 * 15 * 2, "f16": 2 * 15 * 2}
PRECISION_CODE = {"f32": 0, "bf16": 1, "f16": 2}
K3_SOURCE = os.path.join(ROOT, "paper_1909_13412_gb300", "csrc", "lbm_kernels.cu")
# committed ncu summaries with the DRAM bytes per lattice launch at 256^3, per storage type
K3_PROFILE = {"f32": os.path.join(ROOT, "profiles", "stream_collide_forced_256.md"),
              "bf16": os.path.join(ROOT, "profiles", "stream_collide_quad_bf16_256.md")}
VACF_LAG = 5000


# names of the lattice kernel's shapes, in the autotuner's order, and (variant, rows) by name
SHAPE_NAMES = [{0: "1node", 1: "2nodes", 3: "4nodes"}[v] + ("_1row" if r == 1 else f"_{r}rows")
               if v != 2 else "bulk_staged" for v, r in AUTOTUNE_SHAPES]
SHAPES = dict(zip(SHAPE_NAMES, AUTOTUNE_SHAPES))
# the lattice kernel each variant launches when the box holds particles
LATTICE_KERNEL = {0: "k_stream_collide_forced", 1: "k_stream_collide_pair", 2: "k_stream_collide_staged",
                  3: "k_stream_collide_quad"}
L2_BYTES = 129e6  # GB300 L2
LAUNCHES_PER_STEP = 2  # particles, stream-collide
VACF_LAUNCHES = 5      # per block of 64 samples: correlator, chunk sum, MSD scan, MSD diagonals, sums


def workload(name):
    if name.endswith(".json"):
        return wl.load(name)
    return {"brownian_256": wl.BROWNIAN_256, "brownian_128": wl.BROWNIAN_128,
            "brownian_64": wl.BROWNIAN_64, "profile_128": wl.PROFILE_128, "profile_192": wl.PROFILE_192,
            "ensemble_68": wl.ENSEMBLE_68}[name]


def make_handle(lbp, w, precision, seed, vacf_lag):
    """A handle holding workload w: one box, or a batch of boxes for an ensemble
    (per-particle VACF, one particle per replica)."""
    if isinstance(w, wl.Ensemble):
        h = lbp.lbp_create_batch(w.boxes, precision=PRECISION_CODE[precision])
        for b in range(len(w.boxes)):
            pb = w.particles(b)
            lbp.lbp_particles_add_to(h, b, pb.r, pb.V, pb.M, pb.gamma, pb.R)
        lbp.lbp_particles_set_params(h, kT=w.kT, seed=seed)
        lbp.lbp_vacf_configure_ex(h, vacf_lag, 1)
        return h
    nz, ny, nx = w.shape_zyx
    ps = w.particles()
    h = lbp.lbp_create(nx, ny, nz, w.tau, precision=PRECISION_CODE[precision])
    lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
    lbp.lbp_particles_set_params(h, kT=w.kT, seed=seed)
    lbp.lbp_vacf_configure(h, vacf_lag)
    return h


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(values, device, dist=None):
    """Element-wise max of per-rank timings over all ranks (identity when alone)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def aggregate_mlups(world, nodes_per_rank, steps, max_ms):
    """Whole-job lattice updates per second (MLUPS) over `world` replica boxes."""
    return world * nodes_per_rank * steps / (max_ms * 1e-3) / 1e6


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recorded_traffic(precision, shape):
    """DRAM bytes per stream-collide launch from the committed ncu summary, if it
    was taken on the current kernel source and, where it names one, with this
    kernel shape (else None)."""
    path = K3_PROFILE.get(precision)
    if not path or not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    m_b = re.search(r"dram_bytes_per_launch_256:\s*([0-9.eE+]+)", text)
    m_shape = re.search(r"kernel_shape:\s*(\w+)", text)
    if not (m_sha and m_b) or (m_shape and m_shape.group(1) != shape):
        return None
    sha = hashlib.sha256(open(K3_SOURCE, "rb").read()).hexdigest()
    return float(m_b.group(1)) if sha == m_sha.group(1) else None


class ClockSampler:
    """nvidia-smi samples every 20 ms from before the warm-up to after the timed
    passes; each sample carries nvidia-smi's own time stamp (host wall clock), so
    the samples taken inside the timed region can be told apart from the rest."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_ms=20):
        self.index = index
        self.period_ms = period_ms
        self.lines = []  # csv lines
        self.proc = None
        self.windows = []  # (t0, t1) host times of the timed regions

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.first = threading.Event()
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi's start-up (NVML initialisation) can stall the GPU's
            # work for about a second: let it finish before anything is timed
            self.first.wait(timeout=10.0)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.first.set()
        self.first.set()

    def mark(self, t0, t1):
        """A timed region, in host wall-clock seconds (time.time())."""
        self.windows.append((t0, t1))

    @staticmethod
    def _stamp(line):
        import datetime
        try:
            return datetime.datetime.strptime(line.split(",")[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def __exit__(self, *exc):
        if self.proc and self.windows:
            # nvidia-smi's output reaches the pipe in blocks: wait (bounded) until a
            # sample taken after the last timed region has arrived, so that the
            # samples of the regions are not lost when the process is stopped
            end = max(b for _, b in self.windows)
            deadline = time.time() + 3.0
            while time.time() < deadline:
                t = self._stamp(self.lines[-1]) if self.lines else None
                if t is not None and t >= end:
                    break
                time.sleep(0.05)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        """Median SM clock and throttle reasons of the samples taken while a timed
        region ran (the nearest sample after each region's start counts too, so a
        region shorter than the sampling period still has one); the same over the
        whole sampled run (warm-up, timed passes, end-to-end run) for context."""
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                t = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((t, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        pick = set()
        for a, b in self.windows:
            pick.update(i for i, r in enumerate(rows) if a <= r[0] <= b)
            after = [i for i, r in enumerate(rows) if r[0] >= a]
            if after:
                pick.add(after[0])

        def stats(sel):
            sm, mx, reasons = [], None, set()
            for i, (t, mhz, mxv, flags) in enumerate(rows):
                if not sel(i):
                    continue
                sm.append(mhz)
                mx = mxv
                for name, val in zip(names, flags):
                    if val.lower() == "active":
                        reasons.add(name)
            return sm, mx, reasons

        inside = lambda i: i in pick
        sm, mx, reasons = stats(inside)
        sm_all, mx_all, reasons_all = stats(lambda i: True)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx if mx else mx_all,
                "reasons": sorted(reasons), "samples": len(sm), "period_ms": self.period_ms,
                "run": {"sm_mhz": statistics.median(sm_all) if sm_all else None,
                        "reasons": sorted(reasons_all), "samples": len(sm_all)}}


# ---------------------------------------------------------------------------- CPU oracle
def oracle_setup(w, ps):
    import oracle
    nz, ny, nx = w.shape_zyx
    o = oracle.Sim(nx, ny, nz, w.tau)
    o.add_particles(ps.r, ps.V, ps.M, ps.gamma, ps.R)
    o.set_params(kT=w.kT, seed=w.seed_noise)
    return o


def cpu_baseline(w, ps, target_s=10.0):
    import oracle
    o = oracle_setup(w, ps)
    t0 = time.perf_counter()
    o.step(1)  # warm-up (first touch of the arrays)
    t1 = time.perf_counter() - t0
    steps = int(min(50, max(1, target_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    cores = oracle.num_threads()
    # the same on one core (a shorter sample: about a fifth of the time budget)
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        o.step(1)
        t1s = time.perf_counter() - t0
        steps1 = int(min(10, max(1, 0.2 * target_s / max(t1s, 1e-3))))
        t0 = time.perf_counter()
        o.step(steps1)
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    o.close()
    return {"value": w.nodes * steps / dt / 1e6, "unit": "MLUPS", "cores": cores,
            "kind": "oracle",
            "single_core": w.nodes * steps1 / dt1 / 1e6,
            "sample": f"{steps} FP64 oracle steps (after 1 warm-up step) of the {w.name} workload "
                      f"({w.nodes} nodes, {w.n_particles} particles; VACF accumulation not included) "
                      f"on {cores} threads; single_core: {steps1} further steps on one thread"}


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if isinstance(w, wl.Ensemble):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single-box workloads"}))
        return 0
    import oracle
    ps = w.particles()
    o = oracle_setup(w, ps)
    t0 = time.perf_counter()
    o.step(max(1, args.warmup))
    t_warm = (time.perf_counter() - t0) / max(1, args.warmup)
    # bound the timed CPU work to ~2 minutes whatever --steps asks for
    steps = int(max(1, min(args.steps, 120.0 / max(t_warm, 1e-3))))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    o.close()
    value = w.nodes * steps / dt / 1e6
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(w, world),
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{steps} timed FP64 oracle steps of the full {w.name} workload "
                                   f"(after {max(1, args.warmup)} warm-up steps)"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def l2_note(nodes, precision):
    """Whether the step's population traffic needs an L2 flush between steps."""
    buf = 15 * nodes * (4 if precision == "f32" else 2)
    if 2 * buf > L2_BYTES:
        return f"no flush: 2 x {buf / 1e6:.0f} MB population buffers per step exceed the 129 MB L2"
    return f"population buffers (2 x {buf / 1e6:.0f} MB) fit in the 129 MB L2: not an HBM-bound case"


def config_of(w, world, vacf_lag=VACF_LAG, precision="f32"):
    if isinstance(w, wl.Ensemble):
        return {"workload": w.name, "boxes": [list(b) for b in w.boxes], "nodes_per_rank": w.nodes,
                "particles_per_rank": w.n_particles, "kT": w.kT, "M": w.M, "gamma": w.gamma,
                "coupling": "stokeslet", "storage": f"{precision} deviation",
                "vacf_max_lag": vacf_lag, "vacf": "per particle (= per replica)",
                "parallelism": f"replicas{world}",
                "l2": l2_note(w.nodes, precision)}
    nz, ny, nx = w.shape_zyx
    return {"workload": w.name, "lattice": [nx, ny, nz], "nodes_per_rank": w.nodes,
            "particles_per_rank": w.n_particles, "tau": w.tau, "kT": w.kT, "M": w.M,
            "gamma": w.gamma, "coupling": "stokeslet", "storage": f"{precision} deviation",
            "vacf_max_lag": vacf_lag, "parallelism": f"replicas{world}",
            "l2": l2_note(w.nodes, precision)}


# ---------------------------------------------------------------------------- adjoint
ADJ_BYTES_PER_NODE = 3 * 15 * 4  # lam read + populations read + result write, FP32


def adjoint_variant(lbp, torch, w, ps, steps, checkpoint_every, kT, seed):
    """Record `steps` steps with checkpoints, then the reverse sweep of a
    velocity-relaxation loss; times both, and the adjoint lattice kernel."""
    nz, ny, nx = w.shape_zyx
    h = lbp.lbp_create(nx, ny, nz, w.tau)
    lbp.lbp_particles_add(h, ps.r, ps.V, ps.M, ps.gamma, ps.R)
    lbp.lbp_particles_set_params(h, kT=kT, seed=seed)
    n = ps.n
    vt = torch.empty((steps, n, 3), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    lbp.lbp_adjoint_record(h, steps, checkpoint_every, vt, None)
    ev[1].record(stream)
    torch.cuda.synchronize()
    t = torch.arange(1, steps + 1, dtype=torch.float64, device="cuda")
    v0 = torch.tensor(ps.V, device="cuda")
    target = v0[None] * torch.exp(-t * (w.gamma / w.M))[:, None, None]
    g_v = (2.0 / vt.numel()) * (vt - target)  # d/dV of the mean squared deviation
    out = {k: torch.empty(s_, dtype=torch.float64, device="cuda")
           for k, s_ in (("tau", (1,)), ("gamma", (n,)), ("v0", (n, 3)))}
    lbp.lbp_timing_enable(h, True)
    torch.cuda.synchronize()
    ev[2].record(stream)
    lbp.lbp_adjoint_backward(h, steps, g_v.contiguous(), None, out)
    ev[3].record(stream)
    torch.cuda.synchronize()
    adj_ms, adj_n = lbp.lbp_timing_read(h)
    lbp.lbp_timing_enable(h, False)
    lbp.lbp_destroy(h)
    rec_ms, bwd_ms = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    avg = adj_ms / max(adj_n, 1)
    ach = ADJ_BYTES_PER_NODE * w.nodes / (avg * 1e-3) / 1e9
    return {"workload": w.name, "steps": steps, "checkpoint_every": checkpoint_every, "kT": kT,
            "record_ms": rec_ms, "backward_ms": bwd_ms, "backward_over_record": bwd_ms / rec_ms,
            "value": w.nodes * steps / (bwd_ms * 1e-3) / 1e6,
            "unit": "MLUPS (adjoint steps incl. segment replay)",
            "adjoint_lattice_ms": avg, "adjoint_lattice_launches": adj_n,
            "bytes_per_node": ADJ_BYTES_PER_NODE, "achieved_gbs": ach, "frac": ach / measured_peaks()[0],
            "dL_dtau": float(out["tau"][0])}


# ---------------------------------------------------------------------------- GPU run
def run_gpu(args, w):
    import torch
    from paper_1909_13412_gb300 import lbp

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def make(precision, wk=w):
        h = make_handle(lbp, wk, precision, wk.seed_noise + rank, args.vacf_lag)
        if args.kernel_shape:
            # a fixed shape (reproducible profiles: no timing-dependent pick)
            variant, rows = SHAPES[args.kernel_shape]
            lbp.lbp_set_block_shape(h, rows, variant)
            h.tuned = {"variant": args.kernel_shape, "fixed": True}
            return h
        # block shape of the lattice kernel, picked by timing (outside the timed
        # region) after two steps, so that the candidates see this workload's
        # particle forces in the records
        lbp.lbp_step(h, 2)
        rows, variant, tms = lbp.lbp_autotune(h, 10)
        h.tuned = {"variant": SHAPE_NAMES[AUTOTUNE_SHAPES.index((variant, 1 if variant == 2 else rows))],
                   "ms_by_shape": {n: t for n, t in zip(SHAPE_NAMES, tms) if t > 0}}
        return h

    def vacf_flush(h, out):
        """Correlate the samples not yet in a VACF block (lbp_vacf_read flushes
        them) into device buffers: queued on the stream, no host wait."""
        if out["per_particle"]:
            lbp.lbp_vacf_read_per_particle(h, out["csum"], out["counts"])
        else:
            lbp.lbp_vacf_read(h, out["csum"], out["counts"])

    def vacf_out(h, wk):
        pp = isinstance(wk, wl.Ensemble)
        rows = wk.n_particles if pp else 1
        return {"per_particle": pp,
                "csum": torch.empty((rows, args.vacf_lag + 1), dtype=torch.float64, device="cuda"),
                "counts": torch.empty(args.vacf_lag + 1, dtype=torch.int64, device="cuda")}

    def timed(h, wk, steps, warmup, clocks=None):
        """K steps between CUDA events on the caller's stream, on the path users
        run (CUDA-graph replay, no per-launch events), with the VACF blocks of the
        timed samples -- including the last, partial one, flushed before the end
        event -- inside the region.  Then the same K steps once more with the
        library's events around every stream-collide launch, for that kernel's
        average duration (this pass takes the plain-launch path).  Before the W
        warm-up steps, untimed steps for about a second: a GPU that was idle can
        stall for about a second while its clocks and memory state come up, which
        a timed region of a few milliseconds (small K) must not contain."""
        out = vacf_out(h, wk)
        t_spin = time.time()
        while time.time() - t_spin < 1.0:
            lbp.lbp_step(h, 16)
            torch.cuda.synchronize()
        lbp.lbp_step(h, warmup)
        vacf_flush(h, out)  # nothing of the warm-up's VACF work is left pending
        lbp.lbp_check(h)
        stream = torch.cuda.current_stream()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        t0 = time.time()
        start.record(stream)
        lbp.lbp_step(h, steps)
        vacf_flush(h, out)
        end.record(stream)
        barrier()
        if clocks is not None:
            clocks.mark(t0, time.time())
        ms = start.elapsed_time(end)
        lbp.lbp_check(h)
        # instrumented pass: the lattice kernel's own duration
        lbp.lbp_timing_enable(h, True)
        lbp.lbp_step(h, steps)
        vacf_flush(h, out)
        barrier()
        k3_ms, k3_n = lbp.lbp_timing_read(h)
        lbp.lbp_timing_enable(h, False)
        lbp.lbp_check(h)
        return ms, k3_ms / max(k3_n, 1), k3_n

    def run_e2e(h, wk, clocks):
        """End to end through the C ABI with host buffers: per step the external
        forces go host->device and positions + velocities come back (one
        lbp_step_exchange call per step), and at the end the VACF sums (with the
        flush of the last partial block) are read into host memory."""
        n = wk.n_particles
        fext = torch.zeros((n, 3), dtype=torch.float64).pin_memory().numpy()
        r_h = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
        v_h = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
        pp = isinstance(wk, wl.Ensemble)
        cs_h = torch.empty((n if pp else 1, args.vacf_lag + 1), dtype=torch.float64).pin_memory().numpy()
        cnt_h = torch.empty(args.vacf_lag + 1, dtype=torch.int64).pin_memory().numpy()
        read = lbp.lbp_vacf_read_per_particle if pp else lbp.lbp_vacf_read
        e2e_steps = max(3, min(args.steps, 200))
        for _ in range(max(2, args.warmup)):  # warm-up: both buffer parities
            lbp.lbp_step_exchange(h, fext, r_h, v_h)
        read(h, cs_h, cnt_h)
        barrier()
        t0w = time.time()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            # one public call per step: forces in, one step, positions and velocities out
            lbp.lbp_step_exchange(h, fext, r_h, v_h)
        read(h, cs_h, cnt_h)
        barrier()
        e2e_s = time.perf_counter() - t0
        clocks.mark(t0w, time.time())
        e2e_max_s, = max_over_ranks([e2e_s], "cuda", dist)
        value = aggregate_mlups(world, wk.nodes, e2e_steps, e2e_max_s * 1e3)
        return value, e2e_steps, fext, r_h, v_h, (cs_h.nbytes + cnt_h.nbytes) / e2e_steps

    h = make(args.precision)
    tuned = h.tuned
    clk = ClockSampler(local)
    clk.__enter__()
    try:
        ms, k3_one, k3_n = timed(h, w, args.steps, args.warmup, clk)
        ms_max, k3_avg_ms = max_over_ranks([ms, k3_one], "cuda", dist)
        value = aggregate_mlups(world, w.nodes, args.steps, ms_max)
        e2e_value, e2e_steps, fext, r_h, v_h, e2e_d2h = run_e2e(h, w, clk)
    finally:
        clk.__exit__(None, None, None)
    lbp.lbp_check(h)
    lbp.lbp_destroy(h)

    # the other storage types on the same workload (shorter runs)
    variants = {}
    want = (lambda name: not args.variant or name in args.variant)
    if not args.no_variants and not isinstance(w, wl.Ensemble):
        for prec in ("f32", "bf16", "f16"):
            if prec == args.precision or not want(prec):
                continue
            hv = make(prec)
            vsteps = max(1, min(args.steps, 500))
            vms, vk3, _ = timed(hv, w, vsteps, args.warmup)
            vms, vk3 = max_over_ranks([vms, vk3], "cuda", dist)
            lbp.lbp_destroy(hv)
            vach = BYTES_PER_NODE[prec] * w.nodes / (vk3 * 1e-3) / 1e9
            variants[prec] = {"value": aggregate_mlups(world, w.nodes, vsteps, vms), "unit": "MLUPS",
                              "steps": vsteps, "ms_per_step": vms / vsteps,
                              "kernel": LATTICE_KERNEL[SHAPES[hv.tuned["variant"]][0]],
                              "stream_collide_ms": vk3, "achieved_gbs": vach,
                              "frac": vach / measured_peaks()[0],
                              "traffic": recorded_traffic(prec, hv.tuned["variant"]) if w == wl.BROWNIAN_256
                              else None,
                              "bytes_per_node": BYTES_PER_NODE[prec], "autotune": hv.tuned}
    if not args.no_variants and not isinstance(w, wl.Ensemble) and want("batched"):
        # the batched uneven ensemble: one handle, one lattice launch per step
        e = wl.ENSEMBLE_68
        hb = make(args.precision, e)
        bsteps = max(1, min(args.steps, 1000))
        btuned = hb.tuned
        bms, bk3, _ = timed(hb, e, bsteps, args.warmup)
        bms, bk3 = max_over_ranks([bms, bk3], "cuda", dist)
        lbp.lbp_destroy(hb)
        bach = BYTES_PER_NODE[args.precision] * e.nodes / (bk3 * 1e-3) / 1e9
        variants["batched"] = {"workload": e.name, "value": aggregate_mlups(world, e.nodes, bsteps, bms),
                               "unit": "MLUPS", "boxes": len(e.boxes), "nodes": e.nodes,
                               "particles": e.n_particles, "storage": f"{args.precision} deviation",
                               "vacf": f"per particle (= per replica) to lag {args.vacf_lag}",
                               "steps": bsteps, "ms_per_step": bms / bsteps,
                               "stream_collide_ms": bk3, "achieved_gbs": bach,
                               "frac": bach / measured_peaks()[0],
                               "particle_updates_per_s": world * e.n_particles * bsteps / (bms * 1e-3),
                               "autotune": btuned}

    if not args.no_variants and not isinstance(w, wl.Ensemble) and want("adjoint_64"):
        # the differentiable run: 64^3, 8 kicked particles, 2000 steps, checkpoint every 100
        wa = wl.ADJOINT_64
        variants["adjoint_64"] = adjoint_variant(lbp, torch, wa, wl.kicked_particles(wa), wa.steps,
                                                 wa.extra["checkpoint_every"], 0.0, 0)
    if not args.no_variants and not isinstance(w, wl.Ensemble) and want("adjoint"):
        # the reverse sweep on the bench workload itself (population copies larger than L2)
        key = "adjoint_256" if w == wl.BROWNIAN_256 else "adjoint_" + w.name
        variants[key] = adjoint_variant(lbp, torch, w, w.particles(), 100, 20, w.kT, w.seed_noise)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_NODE[args.precision] * w.nodes / (k3_avg_ms * 1e-3) / 1e9
    traffic = recorded_traffic(args.precision, tuned["variant"]) if w == wl.BROWNIAN_256 else None
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(w, world, args.vacf_lag, args.precision),
        "roofline": {"bound": "hbm", "kernel": LATTICE_KERNEL[SHAPES[tuned["variant"]][0]], "achieved": achieved,
                     "peak": peak, "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": BYTES_PER_NODE[args.precision] * w.nodes,
                     "avg_launch_ms": k3_avg_ms, "launches": k3_n},
        "particle_updates_per_s": world * w.n_particles * args.steps / (ms_max * 1e-3),
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": fext.nbytes,
                "d2h_bytes_per_step": r_h.nbytes + v_h.nbytes + e2e_d2h, "steps": e2e_steps,
                "note": "one lbp_step_exchange per step (forces in, positions and velocities out, "
                        "page-locked host buffers), then the VACF sums read to the host"},
        "autotune": tuned,
        "variants": variants,
        # per step the particle kernel and the lattice kernel; per block of 64
        # samples the VACF and MSD kernels (five, or one per-particle VACF
        # kernel), and the same once more for the flush of the last, partial
        # block at the end of the region
        "gpu_launches": LAUNCHES_PER_STEP * args.steps
                        + (1 if isinstance(w, wl.Ensemble) else VACF_LAUNCHES) * (args.steps // 64 + 1),
        "timing": "headline on the graph-replay path without per-launch events; the lattice "
                  "kernel's average from a second, instrumented pass of the same steps",
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline and not isinstance(w, wl.Ensemble):
        line["cpu_baseline"] = cpu_baseline(w, w.particles())
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["lbp", "reference"], default="lbp")
    ap.add_argument("--workload", default="brownian_256",
                    help="brownian_256, brownian_128, brownian_64, profile_128, profile_192, ensemble_68, "
                         "or a workload JSON file (paper_1909_13412_gb300/configs/)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--vacf-lag", type=int, default=VACF_LAG)
    ap.add_argument("--precision", choices=["f32", "bf16", "f16"], default="f32")
    ap.add_argument("--kernel-shape", choices=SHAPE_NAMES, default=None,
                    help="fix the lattice kernel's shape instead of autotuning it")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--variant", action="append", default=[],
                    help="run only these variants (bf16, f16, f32, batched, adjoint_64, adjoint); default all")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "lbp":
        args.warmup = 3
    w = workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, w)
    return run_gpu(args, w)


if __name__ == "__main__":
    sys.exit(main())
