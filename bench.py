"""Benchmark of the peridynamic explicit step: bond updates per second.

One step = one fused force + velocity-Verlet kernel of the whole lattice (PMB),
or the dilatation pass plus the fused force + update kernel (LPS). A bond
update is one directed bond processed in one step, all passes of that step.

Default workload: 3D block 64^3 (h = 1/64 m, m = 3, 30,289,512 directed bonds),
PMB with breaking at s_c = 1e-3, Gaussian velocity pulse and pre-notch,
FP32-compensated bond arithmetic with FP64 integrator state. Its per-step
working set (~45 MB) fits in the 129 MB L2, so L2 is flushed (a 512 MB write,
then a 256 MB read) before every timed step and each step is timed alone with CUDA events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload block64|lps128|plate50]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

Multi-GPU: independent replicas (the step does not shard across GPUs here), one
per rank; value = all ranks' bond updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1806_06917_gb300 import workloads as W  # noqa: E402

SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# FP32 arithmetic of one bond as the kernels evaluate it (hand count; an FMA is
# one operation; the 2 MUFU ops per bond are not included).
# NP in 2D (np_fast): eta 2, S = eta.d/|d|^2 3, t S 1, a S^2 2, times exp 1,
# force 2 (11, plus one MUFU ex2).
FP32_OPS_PER_BOND = {"pmb3": 24, "pmb2": 18, "lps_dil": 19, "lps_force": 30, "np2": 11}
# FP64 path (pmb_generic<double>): the arithmetic of one bond as written, flops
# with an FMA as 2 and rsqrt, divide as one each (their expansion into several
# FP64 instructions is not counted): eta, y 6; |y|^2 5; numerator 10; rsqrt 1;
# stretch 6; weight 1; force 6 (plus 2 for the partial-volume factor when on).
FP64_OPS_PER_BOND = 35
FP64_NOMINAL_TFLOPS = 1.25

# Algorithmic bytes per point of one step, in the kernels' layout (u and v as
# double-float pairs, 2 x float4 = 32 B each): u read 32, v read + written 64,
# new u written 32, bond-mask words read (4 B x W: W = 4 in 3D, 1 in 2D at m = 3,
# 40 in 2D at m = 20), BC kinds 1 B per DOF. LPS: dilatation pass u 32 + masks
# 16 + 1/m~ 4 read, theta 4 written (56); force pass u 32 + theta, 1/m~ 8 +
# masks 16 read, v 64, new u 32, BC kinds 3 (155).
BYTES_PER_POINT = {"pmb3": 147.0, "pmb2": 134.0, "lps": 211.0, "np2": 128.0 + 4 * 40 + 2}
CSR_BYTES_PER_BOND = {"pmb3": 4.25, "pmb2": 4.25, "lps": 8.0, "np2": 4.0}
KERNEL_LABEL = {
    "pmb3": lambda wl: "pmb_fast<3, %s>" % ("true" if wl.mat.s_c > 0 else "false"),
    "pmb2": lambda wl: "pmb_fast<2, %s>" % ("true" if wl.mat.s_c > 0 else "false"),
    "lps": lambda wl: "lps_dil_fast + lps_force_fast (one step)",
    "np2": lambda wl: "np_fast2<false> (two point pairs per thread)",
}

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one step's
# launches, from one `ncu --set full` capture of each workload's kernels (the
# summaries under profiles/). A figure holds only while the kernel's sources and
# build flags hash to the value recorded with it; otherwise traffic is null.
_KERNEL_COMMON = ["paper_1806_06917_gb300/csrc/pd_internal.cuh", "paper_1806_06917_gb300/csrc/pd_tile.cuh",
                  "paper_1806_06917_gb300/csrc/pd_pair.cuh", "paper_1806_06917_gb300/build.py"]
NCU_TRAFFIC = {
    # (kernel key, tile_log2): the capture of that kernel at that tile size
    ("pmb3", 9): {"bytes": 21903616 + 11264, "sha": "fd63c70de79fc282",
                  "sources": ["paper_1806_06917_gb300/csrc/pd_force_pmb.cu"] + _KERNEL_COMMON,
                  "profile": "profiles/pmb_fast_block3d_64.md"},
    ("pmb3", 8): {"bytes": 21968640 + 1280, "sha": "fd63c70de79fc282",
                  "sources": ["paper_1806_06917_gb300/csrc/pd_force_pmb.cu"] + _KERNEL_COMMON,
                  "profile": "profiles/pmb_fast_block3d_64.md"},
    ("lps", 9): {"bytes": (109791488 + 5980928) + (195891200 + 97487872), "sha": "19443b34cf7d882b",
                 "sources": ["paper_1806_06917_gb300/csrc/pd_force_lps.cu"] + _KERNEL_COMMON,
                 "profile": "profiles/lps_block3d_128.md"},
    ("np2", 9): {"bytes": 45662464 + 73728, "sha": "fd63c70de79fc282",
                 "sources": ["paper_1806_06917_gb300/csrc/pd_force_pmb.cu"] + _KERNEL_COMMON,
                 "profile": "profiles/np_fast2_paper443.md"},
}


def ncu_traffic(key, tile_log2):
    """Bytes per step from the recorded ncu capture of this kernel at this tile
    size, or None if there is none or the kernel changed since."""
    import hashlib
    rec = NCU_TRAFFIC.get((key, tile_log2))
    if rec is None:
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return rec["bytes"] if h.hexdigest()[:16] == rec["sha"] else None


def workload(name):
    if name == "block64":
        wl = W.block3d_pulse(nside=64)
        return wl, "block3d_64_pmb_break: 64^3 lattice, h=1/64 m, m=3, PMB s_c=1e-3, pulse + pre-notch"
    if name == "block256":
        wl = W.block3d_pulse(nside=256)
        return wl, ("block3d_256_pmb_break: 256^3 lattice (16.8M points), h=1/256 m, m=3, PMB s_c=1e-3, "
                    "pulse (w = 8h) + pre-notch; the 64^3 workload at 64x the points")
    if name == "lps128":
        wl = W.block3d_lps(nside=128)
        return wl, "block3d_128_lps: 128^3 lattice, h=1/128 m, m=3, LPS K=40 GPa mu=30 GPa"
    if name == "paper443":
        wl = W.np_benchmark()
        return wl, ("np_benchmark_443_m20: the explicit benchmark shape of Sec. 6.2, 443^2 lattice (196,249 "
                    "nodes), h = 0.0025 m, delta = 0.05 m (m = 20), NP law (C = beta = rho = 1), IC 1 "
                    "Gaussian, collar u = 0, dt = 1e-5")
    if name == "plate50":
        wl = W.plate2d(nside=50)
        return wl, "plate2d_50_pmb: 50^2 lattice, h=0.02 m, m=3, PMB, collar velocities"
    raise SystemExit("unknown workload " + name)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples: a scratch file (the JSON line carries their summary);
        # PD_CLOCKS_DIR keeps them elsewhere
        self.path = os.path.join(os.environ.get("PD_CLOCKS_DIR") or tempfile.gettempdir(),
                                 "pd_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            self.proc.wait(timeout=5)
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ several ranks
# One process per GPU (torchrun). The explicit step does not shard: every rank
# runs its own replica, and ranks meet only to take the slowest rank's time.
# The request mix does shard: rank r serves requests r, r + N, r + 2N, ...


def rank_reduce(torch, x: float, op: str, device: str) -> float:
    """x reduced over the ranks (op "max" or "sum"); x itself on one rank."""
    if not torch.distributed.is_initialized() or torch.distributed.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX if op == "max" else torch.distributed.ReduceOp.SUM)
    return float(t.item())


def shard(items, rank: int, world: int):
    """This rank's share of independent work units (round robin)."""
    return items[rank::world]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh)
    return None


def make_sim(pd, wl, precision, stream, integrator=0, tile_log2=None):
    """The workload's simulation; tile_log2 None picks the tile with pd_tune_tile
    (best of 3 x 10 back-to-back steps per admissible tile), 0 the library default."""
    if tile_log2 is None:
        g, m, r = pd.describe(wl.grid, wl.mat, precision=precision, dt=wl.dt, integrator=integrator)
        tile_log2 = pd.pd_tune_tile(g, m, r, steps=10, stream=stream)
    g, m, r = pd.describe(wl.grid, wl.mat, precision=precision, dt=wl.dt, integrator=integrator,
                          tile_log2=tile_log2)
    sim = pd.pd_create(g, m, r)
    sim.tile_log2 = tile_log2 if tile_log2 else None
    pd.pd_build_neighbors(sim, stream)
    if wl.notch is not None:
        pd.pd_break_bonds(sim, wl.notch.axis, wl.notch.pos, np.asarray(wl.notch.lo), np.asarray(wl.notch.hi),
                          stream)
    return sim


def time_steps(pd, torch, sim, wl, steps, warmup, stream, flush):
    """Per-step CUDA-event durations (ms), L2 flushed before each timed step."""
    pd.pd_set_state(sim, u=wl.u0, v=wl.v0, stream=stream)
    if wl.bc_kind is not None and wl.bc_kind.any():
        pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val, stream)
    pd.pd_step_explicit(sim, warmup, stream)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    half = flush.numel() // 2
    for a, b in evs:
        # flush: write the whole buffer (larger than L2), then read half of it so
        # that the dirty lines are written back before the timed kernel starts
        flush.zero_()
        flush[:half].sum()
        a.record(stream)
        pd.pd_step_explicit(sim, 1, stream)
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def time_build(pd, torch, wl, stream, reps=3):
    """Wall time of pd_build_neighbors (CSR + bond mask + weighted volume + step
    bound, with its allocations and host synchronisations), best of reps after
    one untimed build."""
    g, m, r = pd.describe(wl.grid, wl.mat, precision=pd.PD_FP32C)
    sim = pd.pd_create(g, m, r)
    pd.pd_build_neighbors(sim, stream)
    best = None
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pd.pd_build_neighbors(sim, stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    nb = pd.pd_bond_count(sim)
    sim.close()
    return {"ms": best * 1e3, "bonds": nb, "bonds_per_s": nb / best}


def time_implicit(pd, torch, krylov, precision, nx=200, tangent=None, precond=0):
    """The 200 x 200 clamped plate (left collar u = 0, right collar u_x = 1e-4 W)
    in 10 load steps, one pd_solve_static per step (matrix-free Newton-Krylov,
    linear rtol 1e-8). Wall time of the whole load path and the iteration counts."""
    L = W.plate_static(nx=nx, variant="clamped")
    g, m, r = pd.describe(L.grid, L.mat, precision=precision)
    sim = pd.pd_create(g, m, r)
    pd.pd_build_neighbors(sim)
    z = np.zeros((L.grid.npoints, 2))
    pd.pd_set_state(sim, u=z, v=z)
    fp64 = precision == pd.PD_FP64
    opts = pd.newton_opts(krylov=krylov, restart=50, linear_rtol=1e-8, newton_rtol=1e-8 if fp64 else 1e-6,
                          max_newton_iters=20 if fp64 else 8,
                          tangent=pd.PD_TANGENT_CACHED if tangent is None else tangent, precond=precond)
    newton = lin = conv = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(1, L.load_steps + 1):
        pd.pd_set_bc(sim, L.bc_kind, L.bc_val * s / L.load_steps)
        st = pd.pd_solve_static(sim, opts)
        newton += st["newton_iters"]
        lin += st["linear_iters"]
        conv += st["converged"]
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    nb = pd.pd_bond_count(sim)
    sim.close()
    return {"sec": sec, "load_steps": L.load_steps, "converged_steps": conv, "newton_iters": newton,
            "krylov_iters": lin, "ms_per_krylov_iter": 1e3 * sec / max(lin, 1),
            "tangent_bond_applications_per_s": nb * lin / sec, "bonds": nb}


def time_jvp(pd, torch, precision, nx=200, reps=20):
    """One pd_jvp (user-order device tensors in and out, so the permutation
    kernels are included) on the 200 x 200 plate at a random state; CUDA events."""
    L = W.plate_static(nx=nx, variant="clamped")
    g, m, r = pd.describe(L.grid, L.mat, precision=precision)
    sim = pd.pd_create(g, m, r)
    pd.pd_build_neighbors(sim)
    rng = np.random.default_rng(4)
    u = torch.tensor(rng.normal(0.0, 1e-4 * L.grid.h, (L.grid.npoints, 2)), device="cuda")
    w = torch.tensor(rng.normal(size=(L.grid.npoints, 2)), device="cuda")
    out = torch.empty_like(w)
    pd.pd_set_state(sim, u=u)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        pd.pd_jvp(sim, w, out=out, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        pd.pd_jvp(sim, w, out=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nb = pd.pd_bond_count(sim)
    sim.close()
    return {"ms": ms, "bonds": nb, "bond_applications_per_s": nb / (ms * 1e-3)}


def _submit_request(pd, srv, r):
    g, m, run = pd.describe(r.grid, r.mat, precision=pd.PD_FP32C)
    return pd.pd_submit(srv, g, m, run, r.steps, u0=r.u0)


def run_serving(args, pd, torch, rank=0, world=1):
    """The request mix through the server: one-at-a-time capacity on a sample
    (max_active = 1), then the whole mix arriving as a Poisson process at
    args.load x that capacity, max_active concurrent simulations. With N ranks
    each serves its round-robin share of the mix (arrivals at N x the rate of
    one rank's share), with no collective until the totals are combined."""
    mix = shard(W.serving_mix(count=args.requests), rank, world)
    k = min(args.serial_sample, len(mix))
    srv = pd.Server(max_active=1, quantum_steps=64)
    _submit_request(pd, srv, mix[0])                       # warm-up (module load, first graph)
    t0 = time.perf_counter()
    sres = [pd.pd_wait(srv, _submit_request(pd, srv, r), timeout_s=600.0) for r in mix[:k]]
    serial_s = time.perf_counter() - t0
    srv.close()
    serial_work = sum(x["bonds"] * r.steps for x, r in zip(sres, mix[:k]))
    capacity = k / serial_s
    # the shard holds every world-th arrival of the global process, so the global
    # rate world x load x capacity offers each rank load x its own capacity
    rate = world * args.load * capacity
    srv = pd.Server(max_active=args.max_active, quantum_steps=args.quantum)
    with Clocks(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        tickets = []
        for r in mix:
            delay = t0 + r.arrival / rate - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(_submit_request(pd, srv, r))
        res = [pd.pd_wait(srv, t, timeout_s=3600.0) for t in tickets]
    srv.close()
    ok = all(x["state"] == pd.PD_REQ_DONE for x in res)
    work = rank_reduce(torch, float(sum(x["bonds"] * r.steps for x, r in zip(res, mix))), "sum", "cuda")
    makespan = rank_reduce(torch, max(x["end_s"] for x in res) - min(x["submit_s"] for x in res), "max", "cuda")
    lat = np.array([x["end_s"] - x["submit_s"] for x in res])
    if world > 1:
        parts = [None] * world
        torch.distributed.all_gather_object(parts, lat.tolist())
        lat = np.array([x for part in parts for x in part])
        ok = bool(rank_reduce(torch, 1.0 if ok else 0.0, "sum", "cuda") == world)
    if rank != 0:
        return
    line = {"metric": "aggregate bond updates/s (served request mix)", "value": work / makespan,
            "unit": "bond-updates/s", "n_gpus": world, "steps": len(lat), "warmup": 1,
            "ms_per_step": 1e3 * makespan / len(lat), "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32 (bond sums), f32 pairs as double-float (integrator state)",
            "data": "synthetic",
            "config": {"workload": "serving_mix: %d requests (2D/3D, PMB/LPS, lognormal sides 20..96, "
                                   "m in {2,3,4}, 100..2000 steps), Poisson arrivals at %.2fx the "
                                   "one-at-a-time capacity" % (args.requests, args.load),
                       "parallelism": "requests sharded round robin over %d rank(s)" % world,
                       "max_active": args.max_active, "quantum_steps": args.quantum, "l2": "not flushed (independent "
                       "simulations stream through it)"},
            "all_done": ok, "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)), "makespan_s": makespan,
            "offered_rate_per_s": rate, "bond_updates": work,
            "serial": {"requests": k, "value": serial_work / serial_s, "unit": "bond-updates/s",
                       "capacity_requests_per_s": capacity},
            "gpu_launches": None, "roofline": None, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_convergence(args, pd, torch):
    """Sec. 5.2.2's 2D study: NP and LP, IC 1 and IC 2, meshes h = delta/2,
    delta/4, delta/8 on [-delta, 1 + delta]^2 with the collar held at 0, dt =
    1e-5 to t = 2. Every 0.1 time units the rate
      alpha = (log ||u_1 - u_2|| - log ||u_2 - u_3||) / log 2
    with ||f||^2 = sum over the coarse nodes in [0, 1]^2 of |f|^2 h_1^2 (the
    coarse nodes are nodes of the finer meshes: index 2i and 4i)."""
    ks = (2, 4, 8)
    steps_total = args.conv_steps
    chunk = max(1, steps_total // 20)
    out = {}
    work = 0
    t_all = time.perf_counter()
    for model in (W.NP, W.LP):
        for ic in (1, 2):
            wls = [W.np_square(k=k, model=model, ic=ic) for k in ks]
            sims = []
            for wl in wls:
                g, m, r = pd.describe(wl.grid, wl.mat, precision=pd.PD_FP32C, dt=wl.dt)
                sim = pd.pd_create(g, m, r)
                pd.pd_build_neighbors(sim)
                pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
                pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val)
                sims.append(sim)
            n1 = wls[0].grid.n[0]
            X1 = wls[0].grid.positions()
            inside = np.all((X1 > -1e-9) & (X1 < 1.0 + 1e-9), axis=1)
            h1 = wls[0].grid.h
            rates, times = [], []
            done = 0
            while done < steps_total:
                q = min(chunk, steps_total - done)
                for sim in sims:
                    pd.pd_step_explicit(sim, q)
                done += q
                us = []
                for wl, sim, k in zip(wls, sims, ks):
                    u, _ = pd.pd_get_state(sim, want_v=False)
                    n = wl.grid.n[0]
                    step = k // ks[0]
                    U = u.reshape(n, n, 2)[::step, ::step].reshape(-1, 2)      # the coarse nodes
                    us.append(U[inside])
                e12 = math.sqrt(float(((us[0] - us[1]) ** 2).sum()) * h1 * h1)
                e23 = math.sqrt(float(((us[1] - us[2]) ** 2).sum()) * h1 * h1)
                times.append(done * wls[0].dt)
                rates.append((math.log(e12) - math.log(e23)) / math.log(2.0) if e12 > 0 and e23 > 0 else None)
            for sim, wl in zip(sims, wls):
                work += pd.pd_bond_count(sim) * steps_total
                sim.close()
            out["%s_ic%d" % ("np" if model == W.NP else "lp", ic)] = {
                "t": [round(t, 4) for t in times], "alpha": [None if a is None else round(a, 4) for a in rates]}
    sec = time.perf_counter() - t_all
    line = {"metric": "bond updates/s (2D NP/LP convergence study, 12 runs)", "value": work / sec,
            "unit": "bond-updates/s", "n_gpus": 1, "steps": steps_total, "warmup": 0, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (bond sums), f32 pairs as double-float (integrator state)", "data": "synthetic",
            "config": {"workload": "Sec. 5.2.2: [0,1]^2, delta = 0.1, h = delta/2, delta/4, delta/8, "
                                   "collar u = 0, dt = 1e-5, t in [0, %g]" % (steps_total * 1e-5),
                       "l2": "not flushed"},
            "seconds": sec, "alpha": out, "gpu_launches": None, "roofline": None}
    print(json.dumps(line), flush=True)


def cpu_baseline(wl, target_s=12.0, max_steps=50):
    """The FP64 oracle (as it stands) on the host cores: a bounded number of explicit
    steps of the same workload."""
    from oracle import oracle as O
    t0 = time.time()
    bonds = O.neighbors(wl.grid)
    if wl.notch is not None:
        O.break_notch(wl.grid, bonds, wl.notch)
    dt = wl.dt if wl.dt > 0 else wl.dt_factor * O.stable_dt(wl.grid, wl.mat, bonds)
    st = O.ExplicitState(wl.grid, wl.mat, bonds, wl.u0, wl.v0, wl.bc_kind, wl.bc_val)
    st.run(dt, 1)                                    # computes f^0 and one step
    setup = time.time() - t0
    t1 = time.time()
    st.run(dt, 1)
    one = max(time.time() - t1, 1e-6)
    n = int(max(1, min(max_steps, target_s / one)))
    t2 = time.time()
    st.run(dt, n)
    el = time.time() - t2
    out = {"value": bonds.nbonds * n / el, "unit": "bond-updates/s", "cores": O.num_threads(),
           "kind": "oracle",
           "sample": "%d explicit steps of the full workload (FP64 C oracle, OpenMP over points); "
                     "setup %.1f s not timed" % (n, setup)}
    # the same oracle on one thread, a few steps
    threads = O.num_threads()
    try:
        O.set_num_threads(1)
        t3 = time.time()
        n1 = max(1, min(3, int(target_s / 4 / (one * threads))))
        st.run(dt, n1)
        el1 = time.time() - t3
        out["single_thread"] = {"value": bonds.nbonds * n1 / el1, "steps": n1}
    finally:
        O.set_num_threads(threads)
    return out, bonds.nbonds


def oracle_step_rate(wl, sample, target_s=3.0, max_steps=20):
    """The oracle's explicit-step rate (as it stands, OpenMP over points) on a
    bounded sample workload of the same model and horizon as a side measurement."""
    from oracle import oracle as O
    bonds = O.neighbors(wl.grid)
    if wl.notch is not None:
        O.break_notch(wl.grid, bonds, wl.notch)
    dt = wl.dt if wl.dt > 0 else wl.dt_factor * O.stable_dt(wl.grid, wl.mat, bonds)
    st = O.ExplicitState(wl.grid, wl.mat, bonds, wl.u0, wl.v0, wl.bc_kind, wl.bc_val)
    st.run(dt, 1)
    t1 = time.time()
    st.run(dt, 1)
    one = max(time.time() - t1, 1e-6)
    n = int(max(1, min(max_steps, target_s / one)))
    t2 = time.time()
    st.run(dt, n)
    el = time.time() - t2
    return {"value": bonds.nbonds * n / el, "unit": "bond-updates/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": "%d explicit steps of %s (%d bonds)" % (n, sample, bonds.nbonds)}


def oracle_build_rate(grid, sample):
    """The oracle's cell-list neighbour build on the host cores."""
    from oracle import oracle as O
    t = time.time()
    b = O.neighbors(grid)
    el = time.time() - t
    return {"value": b.nbonds / el, "unit": "bonds/s", "seconds": el, "cores": O.num_threads(), "kind": "oracle",
            "sample": sample}


def oracle_jvp_rate(nx=200, reps=5):
    """The oracle's tangent product on the 200^2 plate: its central directional
    difference of the FP64 force (two force passes per product)."""
    from oracle import oracle as O
    L = W.plate_static(nx=nx, variant="clamped")
    bonds = O.neighbors(L.grid)
    rng = np.random.default_rng(4)
    u = rng.normal(0.0, 1e-4 * L.grid.h, (L.grid.npoints, 2))
    w = rng.normal(size=(L.grid.npoints, 2))
    O.jvp_fd(L.grid, L.mat, bonds, u, w, 1e-6 * L.grid.h)
    t = time.time()
    for _ in range(reps):
        O.jvp_fd(L.grid, L.mat, bonds, u, w, 1e-6 * L.grid.h)
    el = (time.time() - t) / reps
    return {"value": bonds.nbonds / el, "unit": "bond-applications/s", "ms": el * 1e3, "cores": O.num_threads(),
            "kind": "oracle", "sample": "%d products on the full %d^2 plate (central difference of two FP64 force "
                                        "passes)" % (reps, nx)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl, desc = workload(args.workload)
    from oracle import oracle as O
    bonds = O.neighbors(wl.grid)
    if wl.notch is not None:
        O.break_notch(wl.grid, bonds, wl.notch)
    dt = wl.dt if wl.dt > 0 else wl.dt_factor * O.stable_dt(wl.grid, wl.mat, bonds)
    st = O.ExplicitState(wl.grid, wl.mat, bonds, wl.u0, wl.v0, wl.bc_kind, wl.bc_val)
    st.run(dt, max(args.warmup, 1))
    t0 = time.time()
    st.run(dt, args.steps)
    el = time.time() - t0
    val = bonds.nbonds * args.steps / el
    line = {"impl": "reference", "metric": "bond updates/s (explicit step)", "value": val,
            "unit": "bond-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "bonds": bonds.nbonds},
            "cpu_baseline": {"value": val, "unit": "bond-updates/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": "%d explicit steps of the full workload after %d warm-up steps"
                                       % (args.steps, max(args.warmup, 1))},
            "e2e": {"value": val, "unit": "bond-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="block64",
                    choices=["block64", "block256", "lps128", "plate50", "paper443", "serve", "convergence"])
    ap.add_argument("--conv-steps", type=int, default=200000, help="convergence: steps (dt = 1e-5)")
    ap.add_argument("--requests", type=int, default=512, help="serve: requests in the mix")
    ap.add_argument("--load", type=float, default=2.0, help="serve: offered load / one-at-a-time capacity")
    ap.add_argument("--max-active", type=int, default=16, help="serve: concurrent simulations")
    ap.add_argument("--serial-sample", type=int, default=24, help="serve: requests timed one at a time")
    ap.add_argument("--quantum", type=int, default=64, help="serve: steps per scheduling quantum")
    ap.add_argument("--tile-log2", type=int, default=None,
                    help="tile size 2^N of the timed simulation (6..9; 0 = library default); "
                         "by default pd_tune_tile measures and picks it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64-path and LPS side measurements")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1806_06917_gb300 import pd

    if args.workload == "serve":
        run_serving(args, pd, torch, rank, world)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if args.workload == "convergence":
        if rank == 0:
            run_convergence(args, pd, torch)
        return

    wl, desc = workload(args.workload)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sim = make_sim(pd, wl, pd.PD_FP32C, stream, tile_log2=args.tile_log2)
    nbonds = pd.pd_bond_count(sim)
    key = {W.LPS: "lps", W.NP: "np2"}.get(wl.mat.model, "pmb3" if wl.grid.dim == 3 else "pmb2")
    launches_per_step = 2 if key == "lps" else 1

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    with Clocks(local) as clk:
        t_wall = time.time()
        durs = time_steps(pd, torch, sim, wl, args.steps, args.warmup, stream, flush)
        t_wall = time.time() - t_wall
    barrier()
    ms = rank_reduce(torch, float(np.mean(durs)), "max", "cuda")
    value = world * nbonds / (ms * 1e-3)

    # end to end through the public API, host buffers every step: the state
    # (u, v) in from pinned host memory, one explicit step, u back out to pinned
    # host memory (pd_get_state is synchronous)
    u_h = torch.from_numpy(wl.u0).pin_memory()
    v_h = torch.from_numpy(wl.v0).pin_memory()
    u_o = torch.empty_like(u_h).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        pd.pd_set_state(sim, u=u_h, v=v_h, stream=stream)
        pd.pd_step_explicit(sim, 1, stream)
        pd.pd_get_state(sim, u=u_o, stream=stream, want_v=False)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        pd.pd_set_state(sim, u=u_h, v=v_h, stream=stream)
        pd.pd_step_explicit(sim, 1, stream)
        pd.pd_get_state(sim, u=u_o, stream=stream, want_v=False)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = rank_reduce(torch, e0.elapsed_time(e1), "max", "cuda")
    e2e = {"value": world * nbonds * args.steps / (e2e_ms * 1e-3), "unit": "bond-updates/s",
           "h2d_bytes_per_step": (u_h.numel() + v_h.numel()) * 8,
           "d2h_bytes_per_step": u_o.numel() * 8,
           "note": "per step: pd_set_state(u, v) from pinned host + pd_step_explicit(1) + pd_get_state(u) "
                   "to pinned host; L2 not flushed"}

    # roofline of the dominant kernel: FP32 ALU (not HBM) bound
    ops = FP32_OPS_PER_BOND[key] if key != "lps" else FP32_OPS_PER_BOND["lps_dil"] + FP32_OPS_PER_BOND["lps_force"]
    peak = SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    achieved = ops * nbonds / (ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s (FP32 ops)",
                "frac": achieved / peak, "traffic": ncu_traffic(key, sim.tile_log2),
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz, one op per lane per clock",
                "ops_per_bond": ops, "kernel": KERNEL_LABEL[key](wl),
                "launch_ms": ms / launches_per_step if key != "lps" else ms,
                "traffic_note": "bytes per step (all launches of one step) from one ncu capture, "
                                "cold L2; null when the kernel changed since"}
    if roofline["traffic"] is not None:
        # the captured DRAM bytes per step over this run's step time
        roofline["traffic_gbs"] = roofline["traffic"] / (ms * 1e-3) / 1e9
    peaks = measured_peaks()
    if peaks:
        # per-point bytes the fused step must move (the kernels read no neighbour
        # list); and, for context, the bytes a CSR kernel would add (4 B of col
        # per bond per pass plus the breaking bit)
        bytes_pt, csr_b = BYTES_PER_POINT[key], CSR_BYTES_PER_BOND[key]
        roofline["hbm_frac_of_measured"] = (bytes_pt * wl.grid.npoints / (ms * 1e-3) / 1e9) / peaks["hbm_gbs"]
        roofline["hbm_frac_of_measured_csr_equivalent"] = (
            (bytes_pt * wl.grid.npoints + csr_b * nbonds) / (ms * 1e-3) / 1e9) / peaks["hbm_gbs"]
        roofline["hbm_peak_gbs"] = peaks["hbm_gbs"]

    line = {"metric": "bond updates/s (explicit step)", "value": value,
            "unit": "bond-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (bond sums), f32 pairs as double-float (integrator state)", "data": "synthetic",
            "config": {"workload": desc, "bonds": nbonds, "points": wl.grid.npoints,
                       "l2": "flushed before every timed step (512 MB write, then a 256 MB read that writes the dirty lines back)", "parallelism": "replicas",
                       "launches_per_step": launches_per_step,
                       "tile_log2": sim.tile_log2,
                       "tile_choice": "pd_tune_tile (best of 3 x 10 back-to-back steps per tile)" if args.tile_log2 is None
                       else "--tile-log2"},
            "gpu_launches": args.steps * launches_per_step,
            "roofline": roofline, "e2e": e2e}

    if not args.no_extras and rank == 0:
        # the plain all-FP64 GPU path on the same workload
        sim64 = make_sim(pd, wl, pd.PD_FP64, stream)
        d64 = time_steps(pd, torch, sim64, wl, max(3, min(args.steps, 10)), 3, stream, flush)
        ms64 = float(np.mean(d64))
        line["fp64_path"] = {"value": nbonds / (ms64 * 1e-3), "unit": "bond-updates/s", "ms_per_step": ms64,
                             "tile_log2": sim64.tile_log2,
                             "steps": len(d64), "ratio_fp32c_over_fp64": ms64 / ms,
                             "fp64_ops_per_bond": FP64_OPS_PER_BOND,
                             "fp64_tflops": FP64_OPS_PER_BOND * nbonds / (ms64 * 1e-3) / 1e12,
                             "fp64_frac_of_nominal": FP64_OPS_PER_BOND * nbonds / (ms64 * 1e-3) / 1e12
                             / FP64_NOMINAL_TFLOPS,
                             "fp64_peak_source": "nominal GB300 FP64 rate (not measured on this pool)"}
        sim64.close()
        # accuracy of the FP32-compensated path against the all-FP64 GPU path: the
        # same workload from its initial state, the same number of steps
        acc_steps = 200
        acc = []
        for prec in (pd.PD_FP32C, pd.PD_FP64):
            sa = make_sim(pd, wl, prec, stream, tile_log2=0)
            pd.pd_set_state(sa, u=wl.u0, v=wl.v0, stream=stream)
            if wl.bc_kind is not None and wl.bc_kind.any():
                pd.pd_set_bc(sa, wl.bc_kind, wl.bc_val, stream)
            pd.pd_step_explicit(sa, acc_steps, stream)
            ua, va = pd.pd_get_state(sa, stream=stream)
            acc.append((ua, va, pd.pd_get_broken(sa, stream=stream)))
            sa.close()
        (u32, v32, k32), (u64, v64, k64) = acc
        line["fp32c_vs_fp64"] = {
            "steps": acc_steps,
            "u_rel_l2": float(np.linalg.norm(u32 - u64) / max(np.linalg.norm(u64), 1e-300)),
            "v_rel_l2": float(np.linalg.norm(v32 - v64) / max(np.linalg.norm(v64), 1e-300)),
            "broken_fp32c": int(k32.sum()), "broken_fp64": int(k64.sum()),
            "broken_differ": int((k32 != k64).sum())}
        # the same step with the central-difference drift (Eq. (10))
        simcd = make_sim(pd, wl, pd.PD_FP32C, stream, integrator=pd.PD_INTEGRATOR_CD, tile_log2=sim.tile_log2)
        dcd = time_steps(pd, torch, simcd, wl, max(3, min(args.steps, 10)), 3, stream, flush)
        mscd = float(np.mean(dcd))
        line["central_difference"] = {"value": nbonds / (mscd * 1e-3), "unit": "bond-updates/s",
                                      "ms_per_step": mscd, "steps": len(dcd), "ratio_over_verlet": mscd / ms}
        simcd.close()
        if args.workload == "block64":
            wl2, desc2 = workload("lps128")
            sim2 = make_sim(pd, wl2, pd.PD_FP32C, stream)
            d2 = time_steps(pd, torch, sim2, wl2, 10, 3, stream, flush)
            ms2 = float(np.mean(d2))
            nb2 = pd.pd_bond_count(sim2)
            ops2 = FP32_OPS_PER_BOND["lps_dil"] + FP32_OPS_PER_BOND["lps_force"]
            line["lps128"] = {"workload": desc2, "value": nb2 / (ms2 * 1e-3), "unit": "bond-updates/s",
                              "ms_per_step": ms2, "steps": len(d2), "launches_per_step": 2, "tile_log2": sim2.tile_log2,
                              "alu_frac": ops2 * nb2 / (ms2 * 1e-3) / 1e12 / peak}
            sim2.close()
            # the explicit benchmark shape of Sec. 6.2 (443^2 nodes, m = 20, NP law)
            wl3, desc3 = workload("paper443")
            sim3 = make_sim(pd, wl3, pd.PD_FP32C, stream)
            d3 = time_steps(pd, torch, sim3, wl3, 10, 3, stream, flush)
            ms3 = float(np.mean(d3))
            nb3 = pd.pd_bond_count(sim3)
            line["paper443"] = {"workload": desc3, "value": nb3 / (ms3 * 1e-3), "unit": "bond-updates/s",
                                "ms_per_step": ms3, "steps": len(d3), "launches_per_step": 1, "tile_log2": sim3.tile_log2,
                                "alu_frac": FP32_OPS_PER_BOND["np2"] * nb3 / (ms3 * 1e-3) / 1e12 / peak}
            sim3.close()
            # the same PMB workload at 64x the points (256^3, 2.0e9 bonds): many
            # waves of tiles per SM instead of one
            wl4, desc4 = workload("block256")
            sim4 = make_sim(pd, wl4, pd.PD_FP32C, stream)
            d4 = time_steps(pd, torch, sim4, wl4, 10, 3, stream, flush)
            ms4 = float(np.mean(d4))
            nb4 = pd.pd_bond_count(sim4)
            line["block256"] = {"workload": desc4, "value": nb4 / (ms4 * 1e-3), "unit": "bond-updates/s",
                                "ms_per_step": ms4, "steps": len(d4), "bonds": nb4, "tile_log2": sim4.tile_log2,
                                "alu_frac": FP32_OPS_PER_BOND["pmb3"] * nb4 / (ms4 * 1e-3) / 1e12 / peak}
            sim4.close()
            del wl4
            line["neighbour_build"] = {"block64": time_build(pd, torch, wl, stream),
                                       "lps128": time_build(pd, torch, wl2, stream)}
            line["jvp200"] = {"fp64": time_jvp(pd, torch, pd.PD_FP64), "fp32c": time_jvp(pd, torch, pd.PD_FP32C)}
            line["implicit_plate200"] = {
                "workload": "200x200 plate, h = 1/200 m, m = 3, PMB, left collar clamped, right collar "
                            "u_x = 1e-4 W in 10 load steps; matrix-free Newton-Krylov",
                "gmres50_fp64": time_implicit(pd, torch, pd.PD_KRYLOV_GMRES, pd.PD_FP64),
                "gmres50_fp64_jvp_tangent": time_implicit(pd, torch, pd.PD_KRYLOV_GMRES, pd.PD_FP64,
                                                          tangent=pd.PD_TANGENT_JVP),
                "cg_fp64": time_implicit(pd, torch, pd.PD_KRYLOV_CG, pd.PD_FP64),
                "gmres50_fp64_block_jacobi": time_implicit(pd, torch, pd.PD_KRYLOV_GMRES, pd.PD_FP64,
                                                           precond=pd.PD_PRECOND_BLOCK_JACOBI),
                "pcg_fp64_block_jacobi": time_implicit(pd, torch, pd.PD_KRYLOV_CG, pd.PD_FP64,
                                                       precond=pd.PD_PRECOND_BLOCK_JACOBI),
                "cg_fp32c": time_implicit(pd, torch, pd.PD_KRYLOV_CG, pd.PD_FP32C)}

    line["clocks"] = clk.summary()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, _ = cpu_baseline(wl)
        line["cpu_baseline"] = cb
        if "lps128" in line:
            # the oracle beside the side measurements, each on a bounded sample
            line["lps128"]["cpu_baseline"] = oracle_step_rate(
                W.block3d_lps(nside=40), "a 40^3 LPS block (the 128^3 workload's model, moduli and horizon)")
            line["paper443"]["cpu_baseline"] = oracle_step_rate(
                W.np_square(k=20, delta=0.2), "a 141^2 NP square at m = 20 (the 443^2 step's law and horizon, "
                                              "h = 0.01 m)")
            line["neighbour_build"]["block64"]["cpu_baseline"] = oracle_build_rate(
                wl.grid, "cell-list build of the full 64^3 lattice")
            line["jvp200"]["cpu_baseline"] = oracle_jvp_rate()
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
