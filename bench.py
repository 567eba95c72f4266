#!/usr/bin/env python
"""Throughput of the multiblob inertial-coupling step on the dense 128^3 suspension.

Workload: periodic 128^3 MAC grid (h = rho = eta = 1, dt = 0.05), 18,808 filled icosahedra of
vertex radius 2.2h at volume fraction 0.40 (244,504 blobs), seeded FCC start randomised by
hard-sphere Monte Carlo, springs k = 100, blob repulsion k_rep = 100 within r_cut = 1h, body
force 1e-4 sin(2 pi z / L) x_hat.  One step = one full ICM step of every blob and the fluid.

Metric: fluid cell-steps/s (value) and blob-steps/s, FP32 grid path, with the FP64 grid path
reported beside it.  Device time from CUDA events around each step on the library's stream; the
L2 cache is flushed (a 256 MiB write) between timed steps, outside the events.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank runs an independent replica (no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRID_N = 128
METRIC = "fluid cell-steps/s at 128^3 (FP32 grid); blob-steps/s and FP64 beside it"
WORKLOAD = "dense suspension 128^3, a=2.2h, phi=0.40, 18808 particles x 13 blobs"
DENSE128_BLOBS, DENSE128_PARTICLES = 244504, 18808      # the recipe's counts at seed 3

# What bounds each FP64-grid kernel below the HBM roofline (ncu, dense 128^3 workload).
FP64_LIMITERS = {
    "spread": "FP64 shared-memory atomic adds (one per node contribution)",
    "forces": "FP64 arithmetic of the bond and repulsion forces",
    "fluid_x_fwd": "FP32-pipe issue of the double-float FFT arithmetic",
    "fluid_z_solve": "FP32-pipe issue of the double-float FFT arithmetic",
    "fluid_x_inv": "FP32-pipe issue of the double-float FFT arithmetic",
    "interp_correct": "gather latency (L1 sectors per request)",
    "interp_predict": "gather latency (L1 sectors per request)",
}

# Algorithmic bytes moved by each stage per step, per unit:
#   grid real = 4 B (FP32) / 8 B (FP64); half-spectrum complex = 2 reals; blob FP64 vec = 24 B.
def stage_model(n, nb, rsz, ncell, thermal=False):
    """Algorithmic bytes per stage.  FP32 grids (rsz = 4) fuse the next step's predictor into
    the corrector pass, whose grid v^n + v^{n+1} the inverse plane pass writes; FP64 grids
    (rsz = 8) run the predictor as its own pass and the corrector reads v^n and v^{n+1}."""
    N = n ** 3
    grid = 3 * N * rsz                                  # one 3-component grid
    spec = 3 * n * n * (n // 2 + 1) * 2 * rsz           # one 3-component half spectrum
    vec = 24 * nb
    if rsz == 8:
        return {
            "interp_predict": ("hbm", grid + 2 * vec),   # read v^n, q; write q_half
            "bin": ("hbm", vec + 3 * 4 * nb + 4 * 4 * ncell),
            "forces": ("hbm", nb * (24 + 4 + 4 + 2 * 42 / 13 * 12 + 24 + 48)),
            "force_sum": ("hbm", 0),
            "spread": ("hbm", 48 * nb + grid),
            "fluid_stress": ("hbm", 8 * grid if thermal else 0),
            "fluid_x_fwd": ("hbm", 2 * grid + spec),
            "fluid_y_fwd": ("hbm", 0),
            "fluid_z_solve": ("hbm", 2 * spec),
            "fluid_y_inv": ("hbm", 0),
            "fluid_x_inv": ("hbm", spec + grid),        # read spectrum; write v^{n+1}
            "interp_correct": ("hbm", 2 * grid + 3 * vec),   # read v^n, v^{n+1}, q_half, q; write q
        }
    return {
        # the predictor of step n+1 runs inside step n's corrector pass (same gathered nodes)
        "interp_predict": ("hbm", 0),
        "bin": ("hbm", vec + 3 * 4 * nb + 4 * 4 * ncell), # q_half; cell, rank, slot; counts/scan
        # q_half, slot, pid; write F and the (q, F) record.  The icosahedra share one bond
        # pattern, which the springs read once, not per blob (per-blob lists would add
        # 42/13 bonds x 2 ends x (index + rest) = 78 B a blob)
        "forces": ("hbm", nb * (24 + 4 + 4 + 24 + 48)),
        "force_sum": ("hbm", 0),
        "spread": ("hbm", 48 * nb + grid),               # sorted (q, F) records; write f
        # thermal / convective stress (kT > 0 or advection only): write 9 stress grids, read
        # them and f, write f
        "fluid_stress": ("hbm", 3 * grid + 3 * grid + 2 * grid if thermal else 0),
        "fluid_x_fwd": ("hbm", 2 * grid + spec),         # read v, f; write spectrum
        "fluid_y_fwd": ("hbm", 0),                       # no kernel in the three-pass FFT
        "fluid_z_solve": ("hbm", 2 * spec),
        "fluid_y_inv": ("hbm", 0),                       # no kernel in the three-pass FFT
        # read spectrum and v^n; write v^{n+1} and v^n + v^{n+1} (the corrector's grid)
        "fluid_x_inv": ("hbm", spec + 3 * grid),
        # read v^n + v^{n+1}, v^{n+1}, q_half, q; write q^{n+1} and the next q_half
        "interp_correct": ("hbm", 2 * grid + 4 * vec),
    }


def base_config(nb=DENSE128_BLOBS, npart=DENSE128_PARTICLES, world=1):
    """The workload description shared by both arms' JSON lines."""
    return {"workload": WORKLOAD, "grid": "128^3 MAC, h=rho=eta=1, dt=0.05",
            "blobs": nb, "particles": npart, "precision":
            "FP32 grid/spread/interp/FFT; FP64 positions, forces, mean mode",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "flushed between timed steps (256 MiB write outside the events)"}


def reduce_max(x, dist=None, device=None):
    """The largest of the ranks' values (x itself without a process group).  NCCL groups
    reduce on the rank's GPU, gloo groups on the host."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    import torch
    on = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=on)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, steps, world, ms_max):
    """Whole-job throughput: every rank processes `units_per_rank` per step; the job takes the
    slowest rank's time."""
    return world * units_per_rank * steps / (ms_max * 1e-3)


def measured_traffic(stage):
    """DRAM bytes per launch of the stage's kernel from the committed ncu capture
    (profiles/dram_traffic_dense128.txt), or None when its source changed since the capture."""
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "profiles", "dram_traffic_dense128.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) != 5 or f[0] != stage:
            continue
        # the kernel's source files, '+'-separated (the .cu and the headers it includes)
        srcs = [os.path.join(here, x) for x in f[2].split("+")]
        if not all(os.path.exists(x) for x in srcs):
            return None
        h = hashlib.sha256()
        for x in srcs:
            h.update(open(x, "rb").read())
        if h.hexdigest() != f[3]:
            return None
        return int(f[4])
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)      # about half a second of timed steps
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed steps of the FP64 grid variant (default: min(steps, 10))")
    ap.add_argument("--other-steps", type=int, default=20,
                    help="timed steps of the Stokes-limit and fluctuating 256^3 runs (0: skip)")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--stage-json", default=None, help="also write per-stage times here")
    ap.add_argument("--ref-seconds", type=float, default=None,
                    help="at most this many seconds of timed oracle steps in the reference arm "
                         "(default 120)")
    ap.add_argument("--skip-accuracy", action="store_true",
                    help="skip the error of each reported workload against the oracle")
    return ap.parse_args()


# ----------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms during the timed region (the
    timed loop starts once the first sample has arrived)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.perf_counter()
        while not self.samples and time.perf_counter() - t0 < 3.0:
            time.sleep(0.005)
        self.samples.clear()                     # keep only samples from the timed region

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        smax = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(self.samples)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------------------------
def oracle_sample(threads, warmup=1, steps=3, max_seconds=None, spec_s=None):
    """The FP64 CPU oracle, as it stands, on the benchmark's own inputs (the dense 128^3
    suspension): `warmup` untimed steps, then up to `steps` timed steps (fewer if max_seconds
    runs out, at least one), on `threads` host threads.  Returns (cell-steps/s, blob-steps/s,
    steps, seconds, blobs, threads used)."""
    import oracle
    from paper_1407_5600_gb300 import workloads as wl

    spec, s = spec_s if spec_s is not None else wl.dense_suspension(n=GRID_N, seed=3)
    g = oracle.Grid(spec.nx, spec.ny, spec.nz, h=spec.h, rho=spec.rho, eta=spec.eta,
                    dt=spec.dt, mean_mode=spec.mean_mode)
    before = oracle.set_threads(0)
    used = oracle.set_threads(threads)
    try:
        q, v = s.pos, g.zeros()
        for _ in range(warmup):
            q, v = oracle.step(g, 1, q, v, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep,
                               s.r_cut, body=s.body)
        done, t0 = 0, time.perf_counter()
        while done < steps:
            q, v = oracle.step(g, 1, q, v, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep,
                               s.r_cut, body=s.body)
            done += 1
            if max_seconds is not None and time.perf_counter() - t0 >= max_seconds:
                break
        el = time.perf_counter() - t0
    finally:
        oracle.set_threads(before)
    cells = spec.nx * spec.ny * spec.nz
    return cells * done / el, s.n_blobs * done / el, done, el, s.n_blobs, used


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_baseline_record():
    """The oracle on the benchmark's 128^3 inputs, 1 warm-up + 3 timed steps, on all host cores
    and on one."""
    from paper_1407_5600_gb300 import workloads as wl
    spec_s = wl.dense_suspension(n=GRID_N, seed=3)
    nproc = host_cores()
    cps, bps, st, el, nbl, used = oracle_sample(nproc, spec_s=spec_s)
    cps1, bps1, st1, el1, _, _ = oracle_sample(1, spec_s=spec_s)
    return {"value": cps, "unit": "cell-steps/s", "cores": used, "nproc": nproc,
            "kind": "oracle", "blob_steps_per_s": bps,
            "sample": f"the benchmark's own 128^3 inputs ({nbl} blobs): 1 warm-up + {st} timed "
                      f"FP64 oracle steps on {used} threads (OpenMP over independent loops), "
                      f"{el:.1f} s",
            "single_thread": {"value": cps1, "unit": "cell-steps/s", "cores": 1,
                              "blob_steps_per_s": bps1,
                              "sample": f"1 warm-up + {st1} timed steps on one thread, "
                                        f"{el1:.1f} s"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    nproc = host_cores()
    # the benchmark's own 128^3 inputs; W warm-up and up to K timed steps, bounded in time so
    # that the whole run ends within a few minutes whatever --steps asks for
    budget = args.ref_seconds if args.ref_seconds else 120.0
    cps, bps, steps, el, nblobs, used = oracle_sample(
        nproc, warmup=min(args.warmup, 3), steps=max(1, args.steps), max_seconds=budget)
    sample = (f"{steps} FP64 oracle steps of the benchmark's own 128^3 inputs ({nblobs} blobs) "
              f"on {used} host threads after {min(args.warmup, 3)} warm-up steps, {el:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": cps, "unit": "cell-steps/s",
            "n_gpus": args.gpus, "hardware": "host cores only (the oracle uses no GPU)",
            "steps": steps, "warmup": min(args.warmup, 3),
            "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": base_config(),
            "blob_steps_per_s": bps,
            "cpu_baseline": {"value": cps, "unit": "cell-steps/s", "cores": used,
                             "nproc": nproc, "kind": "oracle", "sample": sample},
            "e2e": {"value": cps, "unit": "cell-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------------
def _rel(a, b):
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b)) / (nb if nb > 0 else 1.0)


def _pos_rel(q, q_ref, q0, L):
    """Relative L2 error of the displacement (minimum image)."""
    d = q - q_ref
    d -= L * np.round(d / L)
    r = q_ref - q0
    r -= L * np.round(r / L)
    return float(np.linalg.norm(d) / max(np.linalg.norm(r), 1e-300))


def accuracy_records(mb, wl, stream, dev, spec, s):
    """Error of every reported workload against the FP64 oracle on the same inputs: relative L2
    of the blob displacements, the fluid velocity and the blob velocities after a few steps from
    rest.  The dense 128^3 runs (both grid precisions, both integrators) use the benchmark's own
    inputs; the fluctuating suspension a 64^3 box of its recipe (same a, phi, kT, Philox seed);
    the gap sweep three of its 32 boxes, stepped inside the batched context."""
    import oracle
    oracle.set_threads(host_cores())
    n = spec.nx
    L = np.array([n * spec.h] * 3)
    out = {}

    def gpu_run(desc, sets, nsteps, ext=None, body=None):
        sim = mb.Multiblob(desc, stream=stream, device=dev)
        try:
            for b, sb in enumerate(sets):
                sim.set_particles(b, sb.pos, sb.pid, sb.bonds, sb.rest, sb.k_spring, sb.k_rep,
                                  sb.r_cut)
            e = None if ext is None else sim._dev(ext, sim.torch.float64)
            for _ in range(nsteps):
                mb.step(sim.ctx, 1, e, body)
            q = sim.blob_positions().cpu().numpy()
            v = sim.velocity_field().cpu().numpy().astype(np.float64)
            u = sim.blob_velocities().cpu().numpy()
        finally:
            sim.close()
        return q, v, u

    def ograd(sp, integrator=0):
        return oracle.Grid(sp.nx, sp.ny, sp.nz, h=sp.h, rho=sp.rho, eta=sp.eta, dt=sp.dt,
                           mean_mode=1 if integrator else sp.mean_mode)

    # dense 128^3, ICM, both grid precisions: 3 steps (direct, then graph replays)
    g = ograd(spec)
    q_ref, v_ref = oracle.step(g, 3, s.pos, g.zeros(), s.pid, s.bonds, s.rest, s.k_spring,
                               s.k_rep, s.r_cut, body=s.body)
    u_ref = oracle.interp(g, q_ref, v_ref)
    for prec in (0, 1):
        d = mb.GridDesc(n, n, n, precision=prec, dt=spec.dt, rho=spec.rho, eta=spec.eta,
                        h=spec.h, mean_mode=spec.mean_mode)
        q, v, u = gpu_run(d, [s], 3, body=s.body)
        out["dense128_fp32" if prec == 0 else "dense128_fp64"] = {
            "steps": 3, "q_displacement_rel_l2": _pos_rel(q, q_ref, s.pos, L),
            "v_rel_l2": _rel(v[0], v_ref), "u_rel_l2": _rel(u, u_ref),
            "sample": "the benchmark's own 128^3 inputs, 3 steps from rest"}
    # Stokes limit on the same inputs: 2 steps
    gs = ograd(spec, 1)
    qs_ref, vs_ref = oracle.stokes_step(gs, 2, s.pos, s.pid, s.bonds, s.rest, s.k_spring,
                                        s.k_rep, s.r_cut, body=s.body)
    d = mb.GridDesc(n, n, n, precision=0, dt=spec.dt, eta=spec.eta, h=spec.h, mean_mode=1,
                    integrator=1)
    q, v, _ = gpu_run(d, [s], 2, body=s.body)
    out["stokes_limit_dense128"] = {
        "steps": 2, "q_displacement_rel_l2": _pos_rel(q, qs_ref, s.pos, L),
        "v_rel_l2": _rel(v[0], vs_ref), "sample": "the benchmark's own 128^3 inputs"}
    del q_ref, v_ref, u_ref, qs_ref, vs_ref
    # fluctuating suspension: a 64^3 box of the 256^3 recipe, 2 steps of thermal stress
    spec5, s5 = wl.fluctuating_suspension(n=64, a=3.2, phi=0.30, kT=1e-3, seed=5)
    g5 = ograd(spec5)
    q5_ref, v5_ref = oracle.step(g5, 2, s5.pos, g5.zeros(), s5.pid, s5.bonds, s5.rest,
                                 s5.k_spring, s5.k_rep, s5.r_cut, kT=spec5.kT, seed=17)
    d = mb.GridDesc(64, 64, 64, precision=0, dt=spec5.dt, eta=spec5.eta, h=spec5.h,
                    mean_mode=spec5.mean_mode, kT=spec5.kT, seed=17)
    q, v, u = gpu_run(d, [s5], 2)
    out["fluctuating_256"] = {
        "steps": 2, "q_displacement_rel_l2": _pos_rel(q, q5_ref, s5.pos, np.array([64.0] * 3)),
        "v_rel_l2": _rel(v[0], v5_ref), "u_rel_l2": _rel(u, oracle.interp(g5, q5_ref, v5_ref)),
        "sample": f"64^3 box of the same recipe ({s5.n_blobs} blobs), kT = 1e-3, Philox seed 17"}
    # gap sweep: the batched context of 32 boxes, boxes 0, 15 and 31 against the oracle
    sweep = [wl.gap_sweep_box(b, n_boxes=32, n=64, a=1.6) for b in range(32)]
    spec2 = sweep[0][0]
    d = mb.GridDesc(64, 64, 64, batch=32, precision=0, dt=spec2.dt, eta=spec2.eta, h=spec2.h,
                    mean_mode=spec2.mean_mode)
    ext2 = np.concatenate([sb.ext for _, sb in sweep])
    q, v, u = gpu_run(d, [sb for _, sb in sweep], 2, ext=ext2)
    g2 = ograd(spec2)
    errs = []
    for b in (0, 15, 31):
        sb = sweep[b][1]
        qb_ref, vb_ref = oracle.step(g2, 2, sb.pos, g2.zeros(), sb.pid, sb.bonds, sb.rest,
                                     sb.k_spring, ext=sb.ext)
        sl = slice(26 * b, 26 * b + 26)
        errs.append((_pos_rel(q[sl], qb_ref, sb.pos, np.array([64.0] * 3)),
                     _rel(v[b], vb_ref), _rel(u[sl], oracle.interp(g2, qb_ref, vb_ref))))
    e = np.max(np.array(errs), axis=0)
    out["gap_sweep_32x64"] = {"steps": 2, "q_displacement_rel_l2": float(e[0]),
                              "v_rel_l2": float(e[1]), "u_rel_l2": float(e[2]),
                              "sample": "boxes 0, 15 and 31 of the batched run (largest error)"}
    return out


def run_ours(args):
    import numpy as np
    import torch

    import paper_1407_5600_gb300 as mb
    from paper_1407_5600_gb300 import workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    spec, s = wl.dense_suspension(n=GRID_N, seed=3 + rank)
    n, nb = GRID_N, s.n_blobs
    cells = n ** 3

    def make(prec):
        sim = mb.Multiblob(mb.GridDesc(n, n, n, precision=prec, dt=spec.dt, rho=spec.rho,
                                       eta=spec.eta, h=spec.h, mean_mode=spec.mean_mode),
                           stream=stream, device=dev)
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        return sim

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()

    def timed_steps(sim, K, stage_timing, body=s.body):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
        if stage_timing:
            mb.set_stage_timing(sim.ctx, True)
        l0 = mb.get_launch_count(sim.ctx)
        barrier()
        for i in range(K):
            flush.fill_(i & 0xFF)                     # evict L2 between timed steps
            evs[i][0].record(stream)
            mb.step(sim.ctx, 1, None, body)
            evs[i][1].record(stream)
        barrier()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        launches = mb.get_launch_count(sim.ctx) - l0
        stages = mb.get_stage_times(sim.ctx) if stage_timing else None
        if stage_timing:
            mb.set_stage_timing(sim.ctx, False)
        return ms, launches, stages

    def max_over_ranks(x):
        return reduce_max(x, dist, dev)

    # ---- FP32 grid (the headline): each step replays the library's captured CUDA graph ----
    sim = make(0)
    for _ in range(args.warmup):
        mb.step(sim.ctx, 1, None, s.body)
    clocks = ClockSampler(local)
    clocks.start()
    ms, launches, _ = timed_steps(sim, args.steps, False)
    clocks.stop()
    tile, tile_ms = mb.get_tuning(sim.ctx)
    ms = max_over_ranks(ms)
    ms_step = ms / args.steps
    value = job_rate(cells, args.steps, world, ms)
    blob_value = job_rate(nb, args.steps, world, ms)
    # ---- the same steps with per-stage CUDA events (direct launches) for the roofline -----
    ms_staged, _, stages = timed_steps(sim, args.steps, True)

    # ---- roofline of the dominant kernel -----------------------------------------------
    ncell = (n // 2) ** 3
    model = stage_model(n, nb, 4, ncell)
    per_stage = {k: {"ms_per_step": v[0] / max(v[1], 1)} for k, v in stages.items()}
    # stages that are one kernel (binning and forces are two each)
    single_kernel = [k for k in per_stage if model[k][1] > 0 and k not in ("bin", "forces")]
    dom = max(single_kernel, key=lambda k: per_stage[k]["ms_per_step"])
    peak, peak_kind = peaks()
    for k, d in per_stage.items():
        bound, byts = model[k]
        d["algorithmic_MB"] = byts / 1e6
        d["GBps"] = byts / (d["ms_per_step"] * 1e-3) / 1e9 if d["ms_per_step"] > 0 else None
        d["frac_hbm"] = d["GBps"] / peak if d["GBps"] else None
    achieved = per_stage[dom]["GBps"]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": measured_traffic(dom),
                "algorithmic_bytes": model[dom][1]}
    step_bytes = sum(model[k][1] for k in model)
    step_frac = step_bytes / (ms_step * 1e-3) / 1e9 / peak
    roofline["note"] = ("kernel time from CUDA events recorded by the library around each stage "
                        "in a second timed loop of the same steps (direct launches); traffic = "
                        "ncu DRAM bytes per launch from profiles/dram_traffic_dense128.txt "
                        "(null when the kernel's source changed since that capture)")

    # ---- end to end through the C ABI with pinned host buffers ---------------------------
    ext_h = torch.zeros((nb, 3), dtype=torch.float64).pin_memory().numpy()
    u_h = torch.empty((nb, 3), dtype=torch.float64).pin_memory().numpy()
    K_e2e = max(3, args.steps)

    def e2e_step():
        mb.step(sim.ctx, 1, ext_h, s.body)           # H2D of the step's blob forces
        mb.get_velocities(sim.ctx, blob_vel=u_h)      # D2H of the step's blob velocities

    for _ in range(max(3, args.warmup)):             # warm-up: captures the graph with forces
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(K_e2e):
        e2e_step()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * cells * K_e2e / e2e_s, "unit": "cell-steps/s",
           "h2d_bytes_per_step": int(ext_h.nbytes), "d2h_bytes_per_step": int(u_h.nbytes),
           "blob_steps_per_s": world * nb * K_e2e / e2e_s,
           "note": "mb_step with external blob forces in pinned host memory + mb_get_velocities "
                   "into pinned host memory every step (zero external force in this workload)"}
    sim.close()

    # ---- FP64 grid variant --------------------------------------------------------------
    K64 = args.fp64_steps if args.fp64_steps is not None else min(args.steps, 10)
    fp64 = None
    if K64 > 0:
        sim64 = make(1)
        for _ in range(max(1, min(args.warmup, 3))):
            mb.step(sim64.ctx, 1, None, s.body)
        ms64, _, _ = timed_steps(sim64, K64, False)          # the step as it runs
        _, _, stages64 = timed_steps(sim64, K64, True)       # the same steps, stage by stage
        ms64 = max_over_ranks(ms64)
        sim64.close()
        model64 = stage_model(n, nb, 8, ncell)
        st64 = {}
        for k, v in stages64.items():
            t = v[0] / max(v[1], 1)
            byts = model64[k][1]
            st64[k] = {"ms_per_step": t, "algorithmic_MB": byts / 1e6,
                       "GBps": byts / (t * 1e-3) / 1e9 if t > 0 and byts else None}
            st64[k]["frac_hbm"] = st64[k]["GBps"] / peak if st64[k]["GBps"] else None
        dom64 = max((k for k in st64 if model64[k][1] > 0 and k not in ("bin", "forces")),
                    key=lambda k: st64[k]["ms_per_step"])
        fp64 = {"value": world * cells * K64 / (ms64 * 1e-3), "unit": "cell-steps/s",
                "blob_steps_per_s": world * nb * K64 / (ms64 * 1e-3),
                "ms_per_step": ms64 / K64, "steps": K64,
                "step_hbm_frac": sum(m[1] for m in model64.values())
                / (ms64 / K64 * 1e-3) / 1e9 / peak,
                "roofline": {"bound": "hbm", "kernel": dom64, "achieved": st64[dom64]["GBps"],
                             "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
                             "frac": st64[dom64]["frac_hbm"], "traffic": None,
                             "algorithmic_bytes": model64[dom64][1],
                             "limiter": FP64_LIMITERS.get(dom64)},
                "stages": st64}

    # ---- the other workloads (FP32 grid), for the record: the Stokes limit on the same
    # suspension, the fluctuating 256^3 suspension (kT = 1e-3, five-pass FFT) and the batched
    # gap sweep (32 boxes of 64^3 in one context) ------------------------------------------
    others = None
    if args.other_steps > 0:
        K2 = args.other_steps
        others = {}
        simS = mb.Multiblob(mb.GridDesc(n, n, n, precision=0, dt=spec.dt, eta=spec.eta, h=spec.h,
                                        mean_mode=1, integrator=1), stream=stream, device=dev)
        simS.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        for _ in range(3):
            mb.step(simS.ctx, 1, None, s.body)
        msS, _, _ = timed_steps(simS, K2, False)
        _, _, stS = timed_steps(simS, K2, True)
        simS.close()
        msS = max_over_ranks(msS)
        others["stokes_limit_dense128"] = {
            "value": world * cells * K2 / (msS * 1e-3), "unit": "cell-steps/s",
            "ms_per_step": msS / K2, "steps": K2,
            "stages_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in stS.items()}}
        spec5, s5 = wl.fluctuating_suspension(n=256, a=3.2, phi=0.30, kT=1e-3, seed=5 + rank)
        n5 = spec5.nx
        sim5 = mb.Multiblob(mb.GridDesc(n5, n5, n5, precision=0, dt=spec5.dt, eta=spec5.eta,
                                        h=spec5.h, mean_mode=spec5.mean_mode, kT=spec5.kT,
                                        seed=17 + rank), stream=stream, device=dev)
        sim5.set_particles(0, s5.pos, s5.pid, s5.bonds, s5.rest, s5.k_spring, s5.k_rep,
                           s5.r_cut)
        for _ in range(3):
            mb.step(sim5.ctx, 1, None, None)
        ms5, _, _ = timed_steps(sim5, K2, False, body=None)
        _, _, st5 = timed_steps(sim5, K2, True, body=None)
        sim5.close()
        ms5 = max_over_ranks(ms5)
        others["fluctuating_256"] = {
            "workload": s5.meta["workload"] + f", {s5.n_particles} particles x 13 blobs",
            "value": world * n5 ** 3 * K2 / (ms5 * 1e-3), "unit": "cell-steps/s",
            "blob_steps_per_s": world * s5.n_blobs * K2 / (ms5 * 1e-3),
            "ms_per_step": ms5 / K2, "steps": K2,
            "stages_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in st5.items()}}
        nbx, n2 = 32, 64
        sweep = [wl.gap_sweep_box(b, n_boxes=nbx, n=n2, a=1.6) for b in range(nbx)]
        spec2 = sweep[0][0]
        sim2 = mb.Multiblob(mb.GridDesc(n2, n2, n2, batch=nbx, precision=0, dt=spec2.dt,
                                        eta=spec2.eta, h=spec2.h, mean_mode=spec2.mean_mode),
                           stream=stream, device=dev)
        for b, (_, sb) in enumerate(sweep):
            sim2.set_particles(b, sb.pos, sb.pid, sb.bonds, sb.rest, sb.k_spring)
        ext2 = torch.from_numpy(np.concatenate([sb.ext for _, sb in sweep])).to(dev)
        for _ in range(3):
            mb.step(sim2.ctx, 1, ext2, None)
        evs2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        barrier()
        evs2[0].record(stream)
        mb.step(sim2.ctx, K2, ext2, None)
        evs2[1].record(stream)
        barrier()
        ms2 = max_over_ranks(evs2[0].elapsed_time(evs2[1]))
        nb2 = sum(sb.n_blobs for _, sb in sweep)
        sim2.close()
        others["gap_sweep_32x64"] = {
            "workload": "batched gap sweep: 32 boxes of 64^3, two particles of a = 1.6h each",
            "value": world * nbx * n2 ** 3 * K2 / (ms2 * 1e-3), "unit": "cell-steps/s",
            "blob_steps_per_s": world * nb2 * K2 / (ms2 * 1e-3),
            "ms_per_step": ms2 / K2, "steps": K2,
            "l2": "not flushed: the grids (velocity pair, force, spectrum: ~0.4 GB) exceed L2"}

    # ---- CPU baseline (oracle, rank 0, N = 1 only) ---------------------------------------
    acc = None
    if rank == 0 and not args.skip_accuracy:
        acc = accuracy_records(mb, wl, stream, dev, spec, s)
        if fp64 is not None:
            fp64["error_vs_oracle"] = acc["dense128_fp64"]
        for k in (others or {}):
            if k in acc:
                others[k]["error_vs_oracle"] = acc[k]
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu_baseline:
        cpu = cpu_baseline_record()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(base_config(nb, s.n_particles, world), spread_tile=list(tile)),
            "blob_steps_per_s": blob_value,
            "step_hbm_frac": step_frac,
            "ms_per_step_stage_timed": ms_staged / args.steps,
            "roofline": roofline,
            "error_vs_oracle": acc["dense128_fp32"] if acc else None,
            "stages": per_stage,
            "fp64": fp64,
            "other_workloads": others,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
        if args.stage_json:
            with open(args.stage_json, "w") as f:
                json.dump(line, f, indent=1)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
