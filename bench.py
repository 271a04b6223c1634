"""Benchmark of the peridynamic explicit step: bond updates per second.

One step = the dilatation pass plus the fused force + update kernel (LPS), or
one fused force + velocity-Verlet kernel of the whole lattice (PMB, NP). A
bond update is one directed bond processed in one step, all passes of that
step.

Default workload: 3D block 128^3 (h = 1/128 m, m = 3, 249,027,944 directed
bonds), state-based LPS (K = 40 GPa, mu = 30 GPa), uniform volumetric strain
1e-4 plus a seeded perturbation, FP32-compensated bond arithmetic with FP64
integrator state. L2 is flushed (a 512 MB write, then a 256 MB read) before
every timed step and each step is timed alone with CUDA events; the two passes
are timed the same way through pd_step_explicit_timed for the roofline. Side
measurements: the all-FP64 GPU path, the double-float-state variant, the 64^3
PMB block with breaking, the 443^2 NP shape of Sec. 6.2, the 256^3 PMB block,
the neighbour build, the tangent product, the implicit load path and a
bounded run of the request server.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload lps128|block64|block256|plate50|paper443]
  python bench.py --workload serve | convergence
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

# Algorithmic bytes of one pass as a CSR-driven kernel would move them: the
# neighbour index col (4 B per bond per pass that walks bonds; the breaking bit,
# 1/8 B read and 1/8 B written per bond, for the bond-based step with
# breaking), and per point X 12 B (FP32), u 24 B read (FP64), the new u 24 B
# written, v 48 B read and written, and the LPS scalars theta, m (4-8 B).
#   PMB fused step: 4.25 B/bond + 110 B/point; LPS dilatation: 4 B/bond + 44
#   B/point; LPS force + update: 4 B/bond + 120 B/point.
ALG_BYTES = {"pmb3": (4.25, 110.0), "pmb2": (4.25, 76.0), "lps_dil": (4.0, 44.0), "lps_force": (4.0, 120.0),
             "np2": (4.0, 76.0)}
# Bytes per point the kernels themselves must move (they read a bond mask of 1
# bit per bond, not col): PMB 3D u staging pair read 32, FP64 u and v read and
# written 96, new staging pair 32, 4 mask words 16, BC kinds 3 (179); LPS
# dilatation u pair 32 + masks 16 + 1/m~ 4 read, theta 4 written (56); LPS
# force pass u pair 32 + theta, 1/m~ 8 + masks 16 read, u, v 96, new pair 32,
# kinds 3 (187); 2D PMB: pair 32, u, v 64, new pair 32, mask 4, kinds 2 (134);
# 2D NP at m = 20: the same with 40 mask words (290).
PER_POINT_BYTES = {"pmb3": 179.0, "pmb2": 134.0, "lps_dil": 56.0, "lps_force": 187.0, "np2": 290.0}
PASS_KERNEL = {"pmb3": "pmb_fast<3, *> (fused force + update)", "pmb2": "pmb_fast<2, *> (fused force + update)",
               "lps_dil": "lps_dil_fast2 (dilatation pass)", "lps_force": "lps_force_fast (force + update pass)",
               "np2": "np_fast2 (fused force + update, two point pairs per thread)"}
FALLBACK_HBM_GBS = 6800.0

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# each pass, from one `ncu --set full` capture of that kernel (the summaries
# under profiles/). A figure holds only while the kernel's sources and build
# flags hash to the value recorded with it; otherwise traffic is null.
_KERNEL_COMMON = ["paper_1806_06917_gb300/csrc/pd_internal.cuh", "paper_1806_06917_gb300/csrc/pd_tile.cuh",
                  "paper_1806_06917_gb300/csrc/pd_pair.cuh", "paper_1806_06917_gb300/build.py"]
_LPS_SOURCES = ["paper_1806_06917_gb300/csrc/pd_force_lps.cu", "paper_1806_06917_gb300/csrc/pd_lps_fast.cuh"]
NCU_TRAFFIC = {
    # (pass key, tile_log2): the capture of that kernel at that tile size
    ("lps_dil", 9): {"bytes": 109745408 + 6098176, "sha": "e7864e5b1918a9c7",
                     "sources": _LPS_SOURCES + _KERNEL_COMMON, "profile": "profiles/lps_block3d_128.md"},
    ("lps_force", 9): {"bytes": 230127872 + 123059968, "sha": "e7864e5b1918a9c7",
                       "sources": _LPS_SOURCES + _KERNEL_COMMON, "profile": "profiles/lps_block3d_128.md"},
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


def make_sim(pd, wl, precision, stream, integrator=0, tile_log2=None, state=0):
    """The workload's simulation; tile_log2 None picks the tile with pd_tune_tile
    (best of 3 x 10 back-to-back steps per admissible tile), 0 the library default."""
    if tile_log2 is None:
        g, m, r = pd.describe(wl.grid, wl.mat, precision=precision, dt=wl.dt, integrator=integrator, state=state)
        tile_log2 = pd.pd_tune_tile(g, m, r, steps=10, stream=stream)
    g, m, r = pd.describe(wl.grid, wl.mat, precision=precision, dt=wl.dt, integrator=integrator,
                          tile_log2=tile_log2, state=state)
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


def time_implicit(pd, torch, krylov, precision, nx=200, tangent=None, precond=0, notch=False):
    """The 200 x 200 clamped plate (left collar u = 0, right collar u_x = 1e-4 W)
    in 10 load steps, one pd_solve_static per step (matrix-free Newton-Krylov,
    linear rtol 1e-8). Wall time of the whole load path and the iteration counts.
    notch: the bonds crossing x = (nx/2 - 1/2) h for y in [0, ny/2] h are broken
    first (a crack across half the plate, normal to the load), so that the
    points on its faces keep about half their bonds."""
    L = W.plate_static(nx=nx, variant="clamped")
    g, m, r = pd.describe(L.grid, L.mat, precision=precision)
    sim = pd.pd_create(g, m, r)
    pd.pd_build_neighbors(sim)
    if notch:
        ny = L.grid.n[1]
        pd.pd_break_bonds(sim, 0, nx / 2 - 0.5, [0.0, -1.0, -1.0], [0.0, ny / 2, 1.0])
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


def run_serving(args, pd, torch, rank=0, world=1, emit=True):
    """The request mix through the server: one-at-a-time capacity on a sample
    (max_active = 1), then the whole mix arriving as a Poisson process at
    args.load x that capacity, max_active concurrent simulations. With N ranks
    each serves its round-robin share of the mix (arrivals at N x the rate of
    one rank's share), with no collective until the totals are combined."""
    sides = getattr(args, "serve_sides", "40,20,96").split(",")
    mix = shard(W.serving_mix(count=args.requests, side_median=float(sides[0]), side_lo=int(sides[1]),
                              side_hi=int(sides[2])), rank, world)
    k = min(args.serial_sample, len(mix))
    mode = pd.PD_SERVE_STREAMS if getattr(args, "serve_mode", "packed") == "streams" else pd.PD_SERVE_PACKED
    # one at a time: every request alone, with the simulation's own kernels
    srv = pd.Server(max_active=1, quantum_steps=64, mode=pd.PD_SERVE_STREAMS)
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
    srv = pd.Server(max_active=args.max_active, quantum_steps=args.quantum, mode=mode,
                    pack_max_tiles=getattr(args, "pack_max_tiles", 0),
                    max_queued=getattr(args, "max_queued", 0))
    rejected = 0
    with Clocks(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        tickets = []
        for r in mix:
            delay = t0 + r.arrival / rate - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            try:
                tickets.append((r, _submit_request(pd, srv, r)))
            except pd.PdError as e:                        # back-pressure (max_queued): refused
                if e.code != pd.PD_EBUSY:
                    raise
                rejected += 1
        res = [pd.pd_wait(srv, t, timeout_s=3600.0) for _, t in tickets]
    srv.close()
    mix = [r for r, _ in tickets]                          # the accepted requests
    ok = all(x["state"] == pd.PD_REQ_DONE for x in res)
    failed = [{"request": i, "state": x["state"], "error": x["error"], "message": x["message"],
               "steps_done": x["steps_done"]} for i, x in enumerate(res) if x["state"] != pd.PD_REQ_DONE]
    # the work done: requests that did not finish count with the steps they took
    work = rank_reduce(torch, float(sum(x["bonds"] * (r.steps if x["state"] == pd.PD_REQ_DONE else x["steps_done"])
                                        for x, r in zip(res, mix))), "sum", "cuda")
    makespan = rank_reduce(torch, max(x["end_s"] for x in res) - min(x["submit_s"] for x in res), "max", "cuda")
    lat = np.array([x["end_s"] - x["submit_s"] for x in res])
    if world > 1:
        parts = [None] * world
        torch.distributed.all_gather_object(parts, lat.tolist())
        lat = np.array([x for part in parts for x in part])
        ok = bool(rank_reduce(torch, 1.0 if ok else 0.0, "sum", "cuda") == world)
        rejected = int(rank_reduce(torch, float(rejected), "sum", "cuda"))
    if rank != 0:
        return
    line = {"metric": "aggregate bond updates/s (served request mix)", "value": work / makespan,
            "unit": "bond-updates/s", "n_gpus": world, "steps": len(lat), "warmup": 1,
            "ms_per_step": 1e3 * makespan / len(lat), "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32 bond arithmetic (compensated), f64 integrator state",
            "data": "synthetic",
            "config": {"workload": "serving_mix: %d requests (2D/3D, PMB/LPS, lognormal sides of median %s "
                                   "in %s..%s, m in {2,3,4}, 100..2000 steps), Poisson arrivals at %.2fx the "
                                   "one-at-a-time capacity" % (args.requests, sides[0], sides[1], sides[2],
                                                               args.load),
                       "parallelism": "requests sharded round robin over %d rank(s)" % world,
                       "max_active": args.max_active, "quantum_steps": args.quantum,
                       "mode": getattr(args, "serve_mode", "packed"),
                       "pack_max_tiles": getattr(args, "pack_max_tiles", 0),
                       "max_queued": getattr(args, "max_queued", 0),
                       "l2": "not flushed (independent simulations stream through it)"},
            "all_done": ok, "failed": failed[:8], "rejected": rejected,
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)), "makespan_s": makespan,
            "offered_rate_per_s": rate, "bond_updates": work,
            "serial": {"requests": k, "value": serial_work / serial_s, "unit": "bond-updates/s",
                       "capacity_requests_per_s": capacity},
            "gpu_launches": None, "roofline": None, "clocks": clk.summary()}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def serve_single(pd, mode, steps, quantum, nside=128):
    """One 128^3 LPS request (the headline workload) alone through the request
    server in `mode`: the wall time of a request of `quantum` steps and of one of
    quantum + steps steps, the difference giving the time per step in that mode
    (admission, setup and the result's copy cancel out)."""
    wl = W.block3d_lps(nside=nside)
    secs = []
    for n in (quantum, quantum + steps):
        srv = pd.Server(max_active=1, quantum_steps=quantum, mode=mode)
        g, m, r = pd.describe(wl.grid, wl.mat, precision=pd.PD_FP32C, tile_log2=9)
        res = pd.pd_wait(srv, pd.pd_submit(srv, g, m, r, n, u0=wl.u0), timeout_s=600.0)
        srv.close()
        if res["state"] != pd.PD_REQ_DONE:
            raise RuntimeError("request failed: %s" % res["message"])
        secs.append(res["end_s"] - res["start_s"])
    return {"ms_per_step": 1e3 * (secs[1] - secs[0]) / steps, "steps": steps, "quantum_steps": quantum}


def coarse_nodes(wl, k, k0):
    """Row indices of the coarse mesh's nodes (k = k0) in [0, 1]^2 on the mesh of
    refinement k: the coarse node i is the fine node k / k0 * i (the lattices are
    aligned at -delta)."""
    n = wl.grid.n[0]
    step = k // k0
    idx = np.arange(n * n).reshape(n, n)[::step, ::step].reshape(-1)
    X = wl.grid.positions()[idx]
    inside = np.all((X > -1e-9) & (X < 1.0 + 1e-9), axis=1)
    return idx[inside]


def convergence_norms(us, wls, ks):
    """||u_1 - u_2||, ||u_2 - u_3|| and ||u_3|| of three meshes h1 > h2 > h3
    (h = delta / k), ||f||^2 = sum over the coarse nodes in [0, 1]^2 of |f|^2 h_1^2."""
    h1 = wls[0].grid.h
    cs = [u[coarse_nodes(wl, k, ks[0])] for u, wl, k in zip(us, wls, ks)]
    e12 = math.sqrt(float(((cs[0] - cs[1]) ** 2).sum()) * h1 * h1)
    e23 = math.sqrt(float(((cs[1] - cs[2]) ** 2).sum()) * h1 * h1)
    n3 = math.sqrt(float((cs[2] ** 2).sum()) * h1 * h1)
    return e12, e23, n3


def convergence_rate(us, wls, ks):
    """Sec. 5.2.2's rate from three meshes h1 > h2 > h3 (h = delta / k):
      alpha = (log ||u_1 - u_2|| - log ||u_2 - u_3||) / log 2."""
    e12, e23, _ = convergence_norms(us, wls, ks)
    return (math.log(e12) - math.log(e23)) / math.log(2.0) if e12 > 0 and e23 > 0 else None


def run_convergence(args, pd, torch):
    """Sec. 5.2.2's 2D study: NP and LP, IC 1 and IC 2, meshes h = delta/k on
    [-delta, 1 + delta]^2 with the collar held at 0, dt = 1e-5 to t = 2. Every
    0.1 time units the rate alpha of every three consecutive meshes of
    --conv-meshes (default 2, 4, 8: the paper's three; a fourth, 16, shows how
    the rate depends on the coarsest mesh)."""
    ks = tuple(int(k) for k in args.conv_meshes.split(","))
    prec = pd.PD_FP64 if args.conv_precision == "fp64" else pd.PD_FP32C
    steps_total = args.conv_steps
    chunk = max(1, steps_total // 20)
    out = {}
    work = 0
    t_all = time.perf_counter()
    cases = set(args.conv_cases.split(","))
    for model in (W.NP, W.LP):
        for ic in (1, 2):
            if "%s_ic%d" % ("np" if model == W.NP else "lp", ic) not in cases:
                continue
            wls = [W.np_square(k=k, model=model, ic=ic) for k in ks]
            sims = []
            for wl in wls:
                g, m, r = pd.describe(wl.grid, wl.mat, precision=prec, dt=wl.dt)
                sim = pd.pd_create(g, m, r)
                pd.pd_build_neighbors(sim)
                pd.pd_set_state(sim, u=wl.u0, v=wl.v0)
                pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val)
                sims.append(sim)
            rates = {"%s" % (ks[i:i + 3],): [] for i in range(len(ks) - 2)}
            norms = {"%s" % (ks[i:i + 3],): [] for i in range(len(ks) - 2)}
            times = []
            done = 0
            while done < steps_total:
                q = min(chunk, steps_total - done)
                for sim in sims:
                    pd.pd_step_explicit(sim, q)
                done += q
                us = [pd.pd_get_state(sim, want_v=False)[0] for sim in sims]
                times.append(done * wls[0].dt)
                for i in range(len(ks) - 2):
                    a = convergence_rate(us[i:i + 3], wls[i:i + 3], ks[i:i + 3])
                    rates["%s" % (ks[i:i + 3],)].append(None if a is None else round(a, 4))
                    norms["%s" % (ks[i:i + 3],)].append(
                        ["%.4e" % x for x in convergence_norms(us[i:i + 3], wls[i:i + 3], ks[i:i + 3])])
            for sim in sims:
                work += pd.pd_bond_count(sim) * steps_total
                sim.close()
            out["%s_ic%d" % ("np" if model == W.NP else "lp", ic)] = {"t": [round(t, 4) for t in times],
                                                                       "alpha": rates,
                                                                       "e12_e23_u3": norms}
    sec = time.perf_counter() - t_all
    line = {"metric": "bond updates/s (2D NP/LP convergence study)", "value": work / sec,
            "unit": "bond-updates/s", "n_gpus": 1, "steps": steps_total, "warmup": 0, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 bond arithmetic (compensated), f64 integrator state" if prec == pd.PD_FP32C else "f64",
            "data": "synthetic",
            "config": {"workload": "Sec. 5.2.2: [0,1]^2, delta = 0.1, h = delta/k for k in %s, "
                                   "collar u = 0, dt = 1e-5, t in [0, %g]" % (list(ks), steps_total * 1e-5),
                       "l2": "not flushed"},
            "seconds": sec, "alpha": out, "gpu_launches": None, "roofline": None}
    print(json.dumps(line), flush=True)


def cpu_model():
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip() + " (" + platform.machine() + ")"
    except Exception:
        pass
    return platform.machine()


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
           "cpu": cpu_model(),
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
            "cpu_baseline": {"value": val, "unit": "bond-updates/s", "cores": O.num_threads(), "cpu": cpu_model(), "kind": "oracle",
                             "sample": "%d explicit steps of the full workload after %d warm-up steps"
                                       % (args.steps, max(args.warmup, 1))},
            "e2e": {"value": val, "unit": "bond-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def pass_times(pd, torch, sim, wl, steps, warmup, stream, flush):
    """Per-pass device times (ms) of single explicit steps, L2 flushed before each:
    (first launch, second launch) of every step, from pd_step_explicit_timed's
    CUDA events on the launching stream."""
    pd.pd_set_state(sim, u=wl.u0, v=wl.v0, stream=stream)
    if wl.bc_kind is not None and wl.bc_kind.any():
        pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val, stream)
    pd.pd_step_explicit(sim, warmup, stream)
    torch.cuda.synchronize()
    half = flush.numel() // 2
    out = []
    for _ in range(steps):
        flush.zero_()
        flush[:half].sum()
        torch.cuda.synchronize()
        out.append(pd.pd_step_explicit_timed(sim, 1, stream))
    return out


def e2e_rate(pd, torch, sim, wl, nbonds, steps, warmup, stream, world):
    """End to end through the public API with host buffers every step: the state
    (u, v) in from pinned host memory, one explicit step, u back out to pinned
    host memory. Pipelined (the value): pd_set_state_async, pd_step_explicit and
    pd_get_state_async per step and one pd_io_sync at the end, so the next
    step's upload overlaps this step's compute and download; every step still
    moves its own input and result across the host link. Beside it the
    synchronous loop (pd_set_state, pd_step_explicit, pd_get_state, which
    returns with the result in host memory)."""
    u_h = torch.from_numpy(wl.u0).pin_memory()
    v_h = torch.from_numpy(wl.v0).pin_memory()
    u_o = torch.empty_like(u_h).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def loop(n, pipelined):
        for _ in range(n):
            if pipelined:
                pd.pd_set_state_async(sim, u=u_h, v=v_h, stream=stream)
                pd.pd_step_explicit(sim, 1, stream)
                pd.pd_get_state_async(sim, u=u_o, stream=stream)
            else:
                pd.pd_set_state(sim, u=u_h, v=v_h, stream=stream)
                pd.pd_step_explicit(sim, 1, stream)
                pd.pd_get_state(sim, u=u_o, stream=stream, want_v=False)
        if pipelined:
            pd.pd_io_sync(sim)

    res = {}
    for pipelined in (True, False):
        loop(warmup, pipelined)
        torch.cuda.synchronize()
        e0.record(stream)
        loop(steps, pipelined)
        e1.record(stream)
        torch.cuda.synchronize()
        res[pipelined] = rank_reduce(torch, e0.elapsed_time(e1), "max", "cuda")
    ms = res[True]
    return {"value": world * nbonds * steps / (ms * 1e-3), "unit": "bond-updates/s",
            "h2d_bytes_per_step": (u_h.numel() + v_h.numel()) * 8, "d2h_bytes_per_step": u_o.numel() * 8,
            "ms_per_step": ms / steps,
            "note": "per step: pd_set_state_async(u, v) from pinned host + pd_step_explicit(1) + "
                    "pd_get_state_async(u) to pinned host, pd_io_sync after the last step (the event that "
                    "ends the timed region is recorded after it); L2 not flushed",
            "sync": {"value": world * nbonds * steps / (res[False] * 1e-3), "ms_per_step": res[False] / steps,
                     "note": "pd_set_state + pd_step_explicit(1) + pd_get_state (synchronous) per step"}}


def roofline_of(key, wl, nbonds, passes_ms, step_ms, tile_log2, peaks):
    """Roofline of the dominant launch (the LPS force + update pass, or the fused
    bond-based step) on the algorithmic bytes of a CSR-driven pass, against the
    measured HBM copy peak; the other pass and the whole step beside it."""
    npts = wl.grid.npoints
    hbm = peaks["hbm_gbs"] if peaks else FALLBACK_HBM_GBS
    src = "MEASURED_PEAKS.json hbm_gbs (measured copy)" if peaks else "fallback 6800 GB/s (no measured peak)"
    names = ["lps_dil", "lps_force"] if key == "lps" else [key]
    per = {}
    for i, nm in enumerate(names):
        b_bond, b_pt = ALG_BYTES[nm]
        byts = b_bond * nbonds + b_pt * npts
        gbs = byts / (passes_ms[i] * 1e-3) / 1e9
        per[nm] = {"kernel": PASS_KERNEL[nm], "launch_ms": passes_ms[i], "bytes_per_launch": byts,
                   "bytes_model": "%g B/bond + %g B/point" % (b_bond, b_pt), "achieved_gbs": gbs,
                   "frac": gbs / hbm, "per_point_bytes": PER_POINT_BYTES[nm],
                   "per_point_frac": PER_POINT_BYTES[nm] * npts / (passes_ms[i] * 1e-3) / 1e9 / hbm,
                   "traffic": ncu_traffic(nm, tile_log2)}
        per[nm]["traffic_gbs"] = (per[nm]["traffic"] / (passes_ms[i] * 1e-3) / 1e9
                                  if per[nm]["traffic"] else None)
    dom = per[names[-1]]
    step_bytes = sum(ALG_BYTES[nm][0] * nbonds + ALG_BYTES[nm][1] * npts for nm in names)
    r = {"bound": "hbm", "achieved": dom["achieved_gbs"], "peak": hbm, "unit": "GB/s", "frac": dom["frac"],
         "traffic": dom["traffic"], "traffic_gbs": dom["traffic_gbs"], "kernel": dom["kernel"],
         "launch_ms": dom["launch_ms"],
         "bytes_per_launch": dom["bytes_per_launch"], "bytes_model": dom["bytes_model"],
         "peak_source": src, "passes": per,
         "step": {"bytes": step_bytes, "ms": step_ms, "achieved_gbs": step_bytes / (step_ms * 1e-3) / 1e9,
                  "frac": step_bytes / (step_ms * 1e-3) / 1e9 / hbm},
         "note": "algorithmic bytes of a CSR-driven pass (col 4 B per bond per pass; per point u, v in FP64, "
                 "X, theta and m~); the kernels read a 1-bit-per-bond mask instead of col, so the bytes they "
                 "must move are the per_point_bytes, and their bound is the L1 / shared-memory pipe "
                 "(profiles/); traffic = ncu dram bytes of one launch, null when the kernel changed since"}
    return r


def explicit_measurement(pd, torch, wl, key, args, stream, flush, state, world, with_e2e):
    """Step rate of one workload: every step timed alone (L2 flushed), the passes
    timed alone the same way, and optionally e2e."""
    sim = make_sim(pd, wl, pd.PD_FP32C, stream, tile_log2=args.tile_log2, state=state)
    nbonds = pd.pd_bond_count(sim)
    durs = time_steps(pd, torch, sim, wl, args.steps, args.warmup, stream, flush)
    ms = rank_reduce(torch, float(np.mean(durs)), "max", "cuda")
    pt = pass_times(pd, torch, sim, wl, max(3, min(args.steps, 20)), args.warmup, stream, flush)
    passes = [float(np.mean([p[0] for p in pt])), float(np.mean([p[1] for p in pt]))]
    out = {"sim": sim, "nbonds": nbonds, "ms": ms, "passes_ms": passes}
    if with_e2e:
        out["e2e"] = e2e_rate(pd, torch, sim, wl, nbonds, args.steps, args.warmup, stream, world)
        out["back_to_back"] = back_to_back(pd, torch, sim, wl, nbonds, stream, world)
    return out


def back_to_back(pd, torch, sim, wl, nbonds, stream, world, steps=64):
    """Steps run back to back as a long run does (pd_step_explicit(steps): CUDA
    graphs of 16 steps replayed), L2 not flushed between them. The step's state,
    staging pairs, bond masks and tables are read (and the state written) every
    step: for the 128^3 LPS block about 290 MB per step, more than the 129 MB
    L2; the 64^3 block's fit in it."""
    pd.pd_set_state(sim, u=wl.u0, v=wl.v0, stream=stream)
    if wl.bc_kind is not None and wl.bc_kind.any():
        pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val, stream)
    pd.pd_step_explicit(sim, 33, stream)                  # the first (restart) step and both graph parities
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pd.pd_step_explicit(sim, steps, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = rank_reduce(torch, e0.elapsed_time(e1), "max", "cuda") / steps
    return {"value": world * nbonds / (ms * 1e-3), "unit": "bond-updates/s", "ms_per_step": ms, "steps": steps,
            "note": "pd_step_explicit(%d) timed as one call (graph replays), L2 not flushed between steps" % steps}


def state_variants(pd, torch, wl, stream, flush, tile_log2, steps=100):
    """The double-float-state variant of the FP32C path beside the FP64-state one:
    its step time, and its u, v difference from the FP64-state run after `steps`
    steps of the workload from its initial state."""
    res = {}
    for name, state in (("f64", pd.PD_STATE_F64), ("df", pd.PD_STATE_DF)):
        sim = make_sim(pd, wl, pd.PD_FP32C, stream, tile_log2=tile_log2, state=state)
        d = time_steps(pd, torch, sim, wl, 10, 3, stream, flush)
        pd.pd_set_state(sim, u=wl.u0, v=wl.v0, stream=stream)
        if wl.bc_kind is not None and wl.bc_kind.any():
            pd.pd_set_bc(sim, wl.bc_kind, wl.bc_val, stream)
        pd.pd_step_explicit(sim, steps, stream)
        u, v = pd.pd_get_state(sim, stream=stream)
        res[name] = (float(np.mean(d)), u, v)
        sim.close()
    (m64, u64, v64), (mdf, udf, vdf) = res["f64"], res["df"]
    return {"ms_per_step_f64_state": m64, "ms_per_step_df_state": mdf, "speedup_df_over_f64": m64 / mdf,
            "steps_compared": steps,
            "u_rel_l2_df_vs_f64": float(np.linalg.norm(udf - u64) / max(np.linalg.norm(u64), 1e-300)),
            "v_rel_l2_df_vs_f64": float(np.linalg.norm(vdf - v64) / max(np.linalg.norm(v64), 1e-300))}


# FP64 operations per bond and step of the all-FP64 path, estimated from the bond
# arithmetic of each pass (square root and division counted as one each): the
# bond-based step about 30, the LPS dilatation about 20 and its force pass 35.
FP64_FLOPS_PER_BOND = {"pmb3": 30.0, "pmb2": 30.0, "lps": 55.0, "np2": 30.0}
FP64_NOMINAL_TFLOPS = 1.25


def fp64_path(pd, torch, wl, stream, flush, nbonds, ms32, peak_note=True):
    """The plain all-FP64 GPU path on the same workload, with its FP64 rate
    against GB300's nominal FP64 rate (no measured FP64 peak is available)."""
    sim64 = make_sim(pd, wl, pd.PD_FP64, stream)
    d64 = time_steps(pd, torch, sim64, wl, 5, 3, stream, flush)
    ms64 = float(np.mean(d64))
    tile = sim64.tile_log2
    sim64.close()
    fpb = FP64_FLOPS_PER_BOND[workload_key(wl)]
    tf = fpb * nbonds / (ms64 * 1e-3) / 1e12
    return {"value": nbonds / (ms64 * 1e-3), "unit": "bond-updates/s", "ms_per_step": ms64, "tile_log2": tile,
            "steps": len(d64), "ratio_fp64_over_fp32c": ms64 / ms32,
            "fp64": {"flops_per_bond": fpb, "achieved_tflops": tf, "peak_tflops": FP64_NOMINAL_TFLOPS,
                     "frac": tf / FP64_NOMINAL_TFLOPS, "peak_source": "nominal GB300 FP64 rate"}}


def fp32c_vs_fp64(pd, wl, stream, steps=200):
    """Accuracy of the FP32C path (FP64 state) against the all-FP64 GPU path: the
    same workload from its initial state, the same number of steps."""
    acc = []
    for prec in (pd.PD_FP32C, pd.PD_FP64):
        sa = make_sim(pd, wl, prec, stream, tile_log2=0)
        pd.pd_set_state(sa, u=wl.u0, v=wl.v0, stream=stream)
        if wl.bc_kind is not None and wl.bc_kind.any():
            pd.pd_set_bc(sa, wl.bc_kind, wl.bc_val, stream)
        pd.pd_step_explicit(sa, steps, stream)
        ua, va = pd.pd_get_state(sa, stream=stream)
        acc.append((ua, va, pd.pd_get_broken(sa, stream=stream)))
        sa.close()
    (u32, v32, k32), (u64, v64, k64) = acc
    return {"steps": steps,
            "u_rel_l2": float(np.linalg.norm(u32 - u64) / max(np.linalg.norm(u64), 1e-300)),
            "v_rel_l2": float(np.linalg.norm(v32 - v64) / max(np.linalg.norm(v64), 1e-300)),
            "broken_fp32c": int(k32.sum()), "broken_fp64": int(k64.sum()), "broken_differ": int((k32 != k64).sum())}


def side_step(pd, torch, name, stream, flush, args):
    """A side workload's FP32C step rate with its roofline (FP64 state)."""
    wl, desc = workload(name)
    key = workload_key(wl)
    sim = make_sim(pd, wl, pd.PD_FP32C, stream)
    nb = pd.pd_bond_count(sim)
    d = time_steps(pd, torch, sim, wl, 10, 3, stream, flush)
    ms = float(np.mean(d))
    pt = pass_times(pd, torch, sim, wl, 5, 2, stream, flush)
    passes = [float(np.mean([p[0] for p in pt])), float(np.mean([p[1] for p in pt]))]
    out = {"workload": desc, "value": nb / (ms * 1e-3), "unit": "bond-updates/s", "ms_per_step": ms,
           "steps": len(d), "bonds": nb, "tile_log2": sim.tile_log2,
           "launches_per_step": 2 if key == "lps" else 1,
           "roofline": roofline_of(key, wl, nb, passes, ms, sim.tile_log2, measured_peaks()),
           "back_to_back": back_to_back(pd, torch, sim, wl, nb, stream, 1)}
    sim.close()
    return out, wl


def serving_side(pd, torch, requests=128, load=2.0, max_active=16, quantum=64):
    """A bounded run of the request server beside the headline: the first
    `requests` of the seeded mix arriving as a Poisson process at `load` x the
    one-at-a-time capacity (measured on 12 requests alone), against those
    one-at-a-time launches; the packed kernel, and every request on its own
    stream beside it."""
    class A:
        pass
    out = None
    for mode in ("packed", "streams"):
        a = A()
        a.requests, a.load, a.max_active, a.quantum, a.serial_sample = requests, load, max_active, quantum, 12
        a.serve_mode, a.pack_max_tiles, a.serve_sides, a.max_queued = mode, 0, "40,20,96", 0
        r = run_serving(a, pd, torch, 0, 1, emit=False)
        if out is None:
            out = r
        else:
            out["streams_mode"] = {k: r[k] for k in ("value", "latency_p50_s", "latency_p99_s", "makespan_s",
                                                     "all_done", "failed", "serial")}
    # the 128^3 LPS workload alone through the server, in both modes
    out["single_lps128"] = {"packed": serve_single(pd, pd.PD_SERVE_PACKED, 384, 64),
                            "streams": serve_single(pd, pd.PD_SERVE_STREAMS, 384, 64)}
    return out


def workload_key(wl):
    return {W.LPS: "lps", W.NP: "np2"}.get(wl.mat.model, "pmb3" if wl.grid.dim == 3 else "pmb2")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lps128",
                    choices=["lps128", "block64", "block256", "plate50", "paper443", "serve", "serve1",
                             "convergence"])
    ap.add_argument("--conv-steps", type=int, default=200000, help="convergence: steps (dt = 1e-5)")
    ap.add_argument("--conv-meshes", default="2,4,8", help="convergence: refinements k (h = delta / k)")
    ap.add_argument("--conv-precision", default="fp32c", choices=["fp32c", "fp64"])
    ap.add_argument("--conv-cases", default="np_ic1,np_ic2,lp_ic1,lp_ic2",
                    help="convergence: the (law, initial condition) cases to run")
    ap.add_argument("--requests", type=int, default=512, help="serve: requests in the mix")
    ap.add_argument("--load", type=float, default=2.0, help="serve: offered load / one-at-a-time capacity")
    ap.add_argument("--max-active", type=int, default=16, help="serve: concurrent simulations")
    ap.add_argument("--serial-sample", type=int, default=24, help="serve: requests timed one at a time")
    ap.add_argument("--quantum", type=int, default=64, help="serve: steps per scheduling quantum")
    ap.add_argument("--serve-mode", default="packed", choices=["packed", "streams"],
                    help="serve: the packed kernel, or every request on its own stream")
    ap.add_argument("--pack-max-tiles", type=int, default=0,
                    help="serve, packed mode: larger requests (in 512-point tiles) run on their own stream; "
                         "0 = no limit (every eligible request is packed)")
    ap.add_argument("--max-queued", type=int, default=0,
                    help="serve: back-pressure, refuse submits while this many wait (0 = no limit)")
    ap.add_argument("--serve-sides", default="40,20,96",
                    help="serve: median, smallest and largest side per axis of the mix's lattices")
    ap.add_argument("--tile-log2", type=int, default=None,
                    help="tile size 2^N of the timed simulation (6..9; 0 = library default); "
                         "by default pd_tune_tile measures and picks it")
    ap.add_argument("--state", default="f64", choices=["f64", "df"],
                    help="integrator state of the timed FP32C simulation: FP64 or double-float")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the side measurements")
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
    if args.workload == "serve1":
        # the 128^3 LPS workload alone through the request server (per-step time of
        # the packed kernel or of the simulation's own kernels on its stream)
        if rank == 0:
            mode = pd.PD_SERVE_STREAMS if args.serve_mode == "streams" else pd.PD_SERVE_PACKED
            r = serve_single(pd, mode, args.steps, args.quantum)
            print(json.dumps({"workload": "128^3 LPS request alone through the server", "mode": args.serve_mode,
                              **r}), flush=True)
        return

    wl, desc = workload(args.workload)
    key = workload_key(wl)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    state = pd.PD_STATE_F64 if args.state == "f64" else pd.PD_STATE_DF
    launches_per_step = 2 if key == "lps" else 1

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    with Clocks(local) as clk:
        m = explicit_measurement(pd, torch, wl, key, args, stream, flush, state, world, with_e2e=True)
    barrier()
    sim, nbonds, ms = m["sim"], m["nbonds"], m["ms"]
    value = world * nbonds / (ms * 1e-3)
    peaks = measured_peaks()
    roofline = roofline_of(key, wl, nbonds, m["passes_ms"], ms, sim.tile_log2, peaks)
    state_desc = "f64 integrator state (u, v)" if state == pd.PD_STATE_F64 else \
        "f32 pairs as double-float integrator state (u, v)"
    line = {"metric": "bond updates/s (explicit step)", "value": value,
            "unit": "bond-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 bond arithmetic (compensated), " + state_desc, "data": "synthetic",
            "config": {"workload": desc, "bonds": nbonds, "points": wl.grid.npoints,
                       "l2": "flushed before every timed step (512 MB write, then a 256 MB read that writes the "
                             "dirty lines back)", "parallelism": "replicas",
                       "launches_per_step": launches_per_step, "tile_log2": sim.tile_log2,
                       "tile_choice": "pd_tune_tile (best of 3 x 10 back-to-back steps per tile)"
                       if args.tile_log2 is None else "--tile-log2"},
            "gpu_launches": args.steps * launches_per_step,
            "roofline": roofline, "e2e": m["e2e"], "back_to_back": m["back_to_back"]}
    sim.close()

    # single-GPU side measurements (their own reductions would wait for the other
    # ranks of a multi-GPU run, which do not take part)
    if not args.no_extras and world == 1:
        line["fp64_path"] = fp64_path(pd, torch, wl, stream, flush, nbonds, ms)
        line["state_variants"] = state_variants(pd, torch, wl, stream, flush, args.tile_log2 or 0)
        line["fp32c_vs_fp64"] = fp32c_vs_fp64(pd, wl, stream, steps=100 if key == "lps" else 200)
        if args.workload == "lps128":
            b64, wl64 = side_step(pd, torch, "block64", stream, flush, args)
            b64["fp64_path"] = fp64_path(pd, torch, wl64, stream, flush, b64["bonds"], b64["ms_per_step"])
            b64["fp32c_vs_fp64"] = fp32c_vs_fp64(pd, wl64, stream, steps=200)
            simcd = make_sim(pd, wl64, pd.PD_FP32C, stream, integrator=pd.PD_INTEGRATOR_CD,
                             tile_log2=b64["tile_log2"])
            dcd = time_steps(pd, torch, simcd, wl64, 10, 3, stream, flush)
            simcd.close()
            b64["central_difference"] = {"ms_per_step": float(np.mean(dcd)),
                                         "ratio_over_verlet": float(np.mean(dcd)) / b64["ms_per_step"]}
            line["block64"] = b64
            line["paper443"], _ = side_step(pd, torch, "paper443", stream, flush, args)
            line["block256"], _ = side_step(pd, torch, "block256", stream, flush, args)
            line["neighbour_build"] = {"lps128": time_build(pd, torch, wl, stream),
                                       "block64": time_build(pd, torch, wl64, stream)}
            line["jvp200"] = {"fp64": time_jvp(pd, torch, pd.PD_FP64), "fp32c": time_jvp(pd, torch, pd.PD_FP32C)}
            line["implicit_plate200"] = {
                "workload": "200x200 plate, h = 1/200 m, m = 3, PMB, left collar clamped, right collar "
                            "u_x = 1e-4 W in 10 load steps; matrix-free Newton-Krylov",
                "gmres50_fp64": time_implicit(pd, torch, pd.PD_KRYLOV_GMRES, pd.PD_FP64),
                "cg_fp64": time_implicit(pd, torch, pd.PD_KRYLOV_CG, pd.PD_FP64),
                "pcg_fp64_block_jacobi": time_implicit(pd, torch, pd.PD_KRYLOV_CG, pd.PD_FP64,
                                                       precond=pd.PD_PRECOND_BLOCK_JACOBI),
                "cg_fp32c": time_implicit(pd, torch, pd.PD_KRYLOV_CG, pd.PD_FP32C),
                "notched": {
                    "workload": "the same plate with a crack across half its height at mid-span",
                    "gmres50_fp64": time_implicit(pd, torch, pd.PD_KRYLOV_GMRES, pd.PD_FP64, notch=True),
                    "gmres50_fp64_block_jacobi": time_implicit(pd, torch, pd.PD_KRYLOV_GMRES, pd.PD_FP64,
                                                               precond=pd.PD_PRECOND_BLOCK_JACOBI, notch=True),
                    "cg_fp64": time_implicit(pd, torch, pd.PD_KRYLOV_CG, pd.PD_FP64, notch=True),
                    "pcg_fp64_block_jacobi": time_implicit(pd, torch, pd.PD_KRYLOV_CG, pd.PD_FP64,
                                                           precond=pd.PD_PRECOND_BLOCK_JACOBI, notch=True)}}
            line["serve"] = serving_side(pd, torch)

    line["clocks"] = clk.summary()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, _ = cpu_baseline(wl)
        line["cpu_baseline"] = cb
        if "block64" in line:
            # the oracle beside the side measurements, each on a bounded sample
            line["block64"]["cpu_baseline"] = oracle_step_rate(
                workload("block64")[0], "the full 64^3 PMB workload")
            line["paper443"]["cpu_baseline"] = oracle_step_rate(
                W.np_square(k=20, delta=0.2), "a 141^2 NP square at m = 20 (the 443^2 step's law and horizon, "
                                              "h = 0.01 m)")
            line["neighbour_build"]["block64"]["cpu_baseline"] = oracle_build_rate(
                workload("block64")[0].grid, "cell-list build of the full 64^3 lattice")
            line["jvp200"]["cpu_baseline"] = oracle_jvp_rate()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
