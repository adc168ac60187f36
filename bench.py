#!/usr/bin/env python
"""Benchmark of the quasi-static projection step on GB300.

One step = one qs_step call: stress/STZ predictor, chi update, wall fill,
right-hand side, multigrid solve of the projection system to relative
residual 1e-10 (warm-started), stress correction.  Workload: 256^3 cells,
simple shear with an STZ-active preload, seeded Gaussian chi field (600 K,
30 K, correlation length 4 cells), mixed precision (FP32 V-cycles inside FP64
iterative refinement).  The same steps in plain FP64 and a cold solve of a
random right-hand side are timed beside it.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).

        python bench.py --sweep-only [--n N] [--nz NZ] [--steps K]
times K finest-level FP32 sweeps alone (two per call, random data, one GPU)
and prints their mean duration; the small case for kernel profiles.

        python bench.py --disc [--n 512] [--nz NZ] [--kind 1|2|3] [--steps 20]
friction-welding disc workload (section 5): n x n x nz cells (nz = n by
default; section 5 prints a 768 x 768 x 384 grid), the top wall rotating
inside radius R = L/3 (omega = 2 pi / (1e8 t_s)) and the bottom one fixed
(kind 1), rotating with it (2) or against it (3); dt = 2e4 t_s, chi0 450 K /
15 K / correlation length 5 cells; mixed and FP64 run in lockstep from the
same state; per-step device times and the mixed run's velocity and stress
error against the FP64 run.
"""
from __future__ import annotations

import argparse
import math
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("sec per multigrid solve (rel resid 1e-10) at 256³, mixed vs FP64; "
          "smoother HBM GB/s")
UNIT = "s/solve"
TOL = 1e-10
PRELOAD = 1.2e9       # Pa, uniform sigma_xz at t0: keeps the STZ rate active
INNER = 0             # FP32 V-cycles per refinement step (0: chosen per step)
SMOOTH_BYTES = 36     # algorithmic bytes per node per FP32 sweep: read v, b; write v (9 floats)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--inner", type=int, default=INNER)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-only", action="store_true")
    ap.add_argument("--fused", action="store_true",
                    help="--sweep-only: the fused one-launch finest sweep (MG_FLAG_FUSED_SWEEP)")
    ap.add_argument("--disc", action="store_true")
    ap.add_argument("--dt-ts", type=float, default=2.0e4)
    ap.add_argument("--kind", type=int, default=1, choices=[1, 2, 3],
                    help="disc walls: 1 top only, 2 both faces together, 3 counter-rotating")
    ap.add_argument("--chi", default="450,15,5",
                    help="disc chi0 recipe: mean K, std K, correlation length in cells")
    ap.add_argument("--nz", type=int, default=0)
    ap.add_argument("--c3-steps", type=int, default=50,
                    help="steps of the mixed-vs-FP64 lockstep run from the initial state")
    ap.add_argument("--c2", action="store_true",
                    help="128^3 x 100 FP64 steps on the GPU in lockstep with the CPU oracle")
    ap.add_argument("--preload", type=float, default=None,
                    help="--c2: initial sigma_xz in Pa (0: the literal unstressed start)")
    ap.add_argument("--cpu-report", action="store_true",
                    help="the CPU oracle's complete runs: 32^3 solve, 256^3 cold solve and "
                         "first 5 steps, 512^3 first step")
    ap.add_argument("--grad", action="store_true",
                    help="64^3 x 40 FP64 steps: plastic work forward alone and with dW/dchi0")
    ap.add_argument("--every", type=int, default=8, help="--grad: checkpoint interval")
    ap.add_argument("--explicit", action="store_true",
                    help="explicit method against the quasi-static one on the section-4 "
                         "comparison geometry (64 x 64 x 32)")
    ap.add_argument("--zeta", default="1e4", help="--explicit: comma-separated zeta values")
    ap.add_argument("--t-end", type=float, default=20.0, help="--explicit: end time in t_s")
    ap.add_argument("--advect", action="store_true",
                    help="default line with the stress advection of the general law "
                         "(MG_FLAG_ADVECT_STRESS) on both sides")
    ap.add_argument("--fma-peak", action="store_true",
                    help="measure the FP64 and FP32 FMA rate of the GPU (the FP64 kernels' roofline)")
    return ap.parse_args()


def run_disc(args):
    """Disc-rotation workload, mixed and FP64 in lockstep (one GPU)."""
    import math

    import torch

    from paper_1904_03808_gb300 import MG_FP64, MG_MIXED, Context, make_state
    from paper_1904_03808_gb300 import inputs as I
    n = args.n or 512
    K = args.steps
    cm, cs_, clc = (float(x) for x in args.chi.split(","))
    t_setup = time.time()
    w = I.Workload(n, steps=K, kind=args.kind, chi_mean=cm, chi_std=cs_, lc_cells=clc, seed=5,
                   dt_ts=args.dt_ts, nz=args.nz or None)
    w.omega = 2.0 * math.pi / (1.0e8 * w.ts)
    v0, s0, c0, t0 = w.initial_state()
    t_setup = time.time() - t_setup
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    st = {}
    for name in ("mixed", "fp64"):
        v, sg, c = (torch.from_numpy(a).to(dev) for a in (v0, s0, c0))
        st[name] = (v, sg, c, make_state(v, sg, c, t0))
    del v0, s0, c0
    ctx = {name: Context(w.nx, w.ny, w.nz, w.h, I.TABLE1["K"], w.mu, bc=w.bc_values(),
                         stz=w.stz, precision=prec, max_cycles=100, stream=stream)
           for name, prec in (("mixed", MG_MIXED), ("fp64", MG_FP64))}
    def max_sbar(sig):
        # largest shear stress sqrt(s0:s0 / 2) over the cells
        tr = (sig[0] + sig[1] + sig[2]) / 3.0
        q = sum((sig[a] - tr) ** 2 for a in range(3)) + 2.0 * sum(sig[a] ** 2 for a in (3, 4, 5))
        return float(torch.sqrt(0.5 * q.max()))

    clocks = Clocks(0)
    clocks.start()
    rows, failed = [], None
    for k in range(K):
        row = {"step": k + 1}
        for name in ("mixed", "fp64"):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            status, stats = ctx[name].step(st[name][3], w.dt, TOL, raise_on_error=False)
            e1.record(stream)
            torch.cuda.synchronize()
            row[name + "_ms"] = e0.elapsed_time(e1)
            row[name + "_cycles"] = stats.cycles
            row[name + "_rel_resid"] = stats.rel_resid
            row[name + "_status"] = status
            row[name + "_max_sbar"] = max_sbar(st[name][1])
        for i, key in ((0, "v"), (1, "sigma")):
            a, b = st["mixed"][i], st["fp64"][i]
            row["err_" + key] = float(torch.linalg.vector_norm(a - b) /
                                      torch.linalg.vector_norm(b))
        rows.append(row)
        if row["mixed_status"] or row["fp64_status"]:
            failed = k + 1
            break
    clk = clocks.stop()
    for c in ctx.values():
        c.close()
    ok_rows = [r for r in rows if not (r["mixed_status"] or r["fp64_status"])] or rows
    tail = ok_rows[1:] if len(ok_rows) > 1 else ok_rows
    mix = statistics.mean(r["mixed_ms"] for r in tail)
    f64 = statistics.mean(r["fp64_ms"] for r in tail)
    return {"mode": "disc", "kind": args.kind, "grid": [w.nx, w.ny, w.nz], "steps": K, "dt_ts": args.dt_ts,
            "omega_rad_s": w.omega, "R_over_L": w.R,
            "chi0": "%g K / %g K / l_c = %g cells, seed 5" % (cm, cs_, clc),
            "mixed_ms_per_step": mix, "fp64_ms_per_step": f64, "speedup_mixed": f64 / mix,
            "first_step_ms": {"mixed": rows[0]["mixed_ms"], "fp64": rows[0]["fp64_ms"]},
            "max_err_v": max(r["err_v"] for r in ok_rows),
            "max_err_sigma": max(r["err_sigma"] for r in ok_rows),
            "worst_rel_resid": max(max(r["mixed_rel_resid"], r["fp64_rel_resid"]) for r in ok_rows),
            "max_sbar_pa": max(r["fp64_max_sbar"] for r in rows), "failed_at_step": failed,
            "host_setup_s": t_setup, "clocks": clk, "per_step": rows}


def run_sweeps(args):
    """Finest-level FP32 sweeps in isolation: nx = ny = n, nz (default n) cells."""
    import torch

    from paper_1904_03808_gb300 import MG_MIXED, Context
    from paper_1904_03808_gb300 import inputs as I
    n = args.n or 256
    nz = args.nz or n
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    from paper_1904_03808_gb300.binding import MG_FLAG_FUSED_SWEEP
    ctx = Context(n, n, nz, 2.0e-2 / n, I.TABLE1["K"], I.TABLE1["mu"], precision=MG_MIXED,
                  stream=stream, flags=MG_FLAG_FUSED_SWEEP if args.fused else 0)
    g = torch.Generator(device=dev).manual_seed(5)
    x = torch.rand((3, nz + 1, n, n), device=dev, dtype=torch.float32, generator=g) - 0.5
    b = torch.rand((3, nz + 1, n, n), device=dev, dtype=torch.float32, generator=g) - 0.5
    for _ in range(max(args.warmup, 3)):
        ctx.smooth(0, b, x, 2, False)
    ctx.profile(True)
    clocks = Clocks(0)
    clocks.start()
    for _ in range(args.steps):
        ctx.smooth(0, b, x, 2, False)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sm_ms, sweeps, launches = ctx.profile_read()
    ctx.profile(False)
    ctx.close()
    t = sm_ms / max(sweeps, 1)
    nodes = n * n * (nz - 1)
    return {"mode": "sweep-only", "kernel": "fused" if args.fused else "two-phase",
            "grid": [n, n, nz], "sweeps": sweeps, "sweep_ms": t,
            "achieved_gbs": SMOOTH_BYTES * nodes / (t / 1e3) / 1e9,
            "launches_per_sweep": launches / max(sweeps, 1), "clocks": clk}


def workload(n):
    from paper_1904_03808_gb300 import inputs as I
    return I.Workload(n, steps=50, strain=0.02, preload=PRELOAD, chi_mean=600.0, chi_std=30.0,
                      lc_cells=4.0, seed=3)


def config(w, extra=None):
    c = {"workload": "simple shear %dx%dx%d cells, STZ-active (sigma_xz0 = %.1f GPa), chi0 seeded "
                     "Gaussian field 600 K / 30 K / l_c = 4 cells, dt = 200 t_s, warm-started "
                     "solves to rel. resid 1e-10" % (w.nx, w.ny, w.nz, PRELOAD / 1e9),
         "grid": [w.nx, w.ny, w.nz], "unknowns": 3 * w.nx * w.ny * (w.nz - 1)}
    # v (corners) + sigma and chi (cells), FP64; L2 is 129 MB
    state_gb = 8.0 * (3 * (w.nz + 1) + 7 * w.nz) * w.nx * w.ny / 1e9
    c["l2"] = ("inputs larger than L2 (state %.2f GB, plus the multigrid hierarchy)" % state_gb
               if state_gb > 0.129 else "inputs smaller than L2 (state %.3f GB)" % state_gb)
    if extra:
        c.update(extra)
    return c


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(t, ws, device=None):
    """Largest of the ranks' times t (the whole job waits for the slowest
    replica); t itself with one rank.  Gloo reduces on the host, NCCL on
    `device`."""
    if ws <= 1:
        return t
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else device
    tt = torch.tensor([t], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt)


def per_solve(t_step, ws):
    """Seconds per solve of the whole job: ws replicas each solve once per
    step in t_step (the max over ranks)."""
    return t_step / ws


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None

    def start(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms",
                 "100", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def code_digest(src: bytes) -> str:
    """sha256 of a C/CUDA source with its // comments, trailing blanks and
    empty lines removed: the digest changes with the code, not the comments."""
    import hashlib
    lines = []
    for ln in src.decode().splitlines():
        ln = ln.split("//", 1)[0].rstrip()
        if ln:
            lines.append(ln)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def traffic_per_sweep(n_nodes):
    """DRAM bytes per finest-level sweep from the committed ncu summary, scaled
    by node count, or None when the smoother code changed since capture."""
    p = os.path.join(ROOT, "profiles", "smoother_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    src = open(os.path.join(ROOT, "paper_1904_03808_gb300", "csrc", d["source"]), "rb").read()
    if code_digest(src) != d["code_sha256"]:
        return None
    return d["dram_bytes_per_node_per_sweep"] * n_nodes


# --------------------------------------------------------------------- oracle

def oracle_step(w, mg, v, sig, chi, t, tol=TOL, advect=False):
    """One complete FP64 CPU oracle qs_step in place (predictor, chi update,
    walls, right-hand side, warm-started multigrid solve to tol, stress
    correction), timed end to end; returns (seconds, V-cycles)."""
    import oracle as O
    t0 = time.perf_counter()
    st, cyc, _ = O.qs_step(mg, v, sig, chi, w.h, w.dt, w.lam, w.mu, O.STZ(**w.stz),
                           O.BC(**w.bc_values()), t, tol=tol, max_cycles=100, advect=advect)
    dt = time.perf_counter() - t0
    if st != 0:
        raise RuntimeError("oracle qs_step failed with status %d" % st)
    return dt, cyc


def oracle_touch(w, mg, v, sig, chi, t):
    """A bounded pass over every array of a step (the pointwise pieces and one
    V-cycle) without advancing the state: the reference arm's warm-up."""
    import oracle as O
    p = O.STZ(**w.stz)
    ss, D, sb = O.stress_star(v, sig, chi, w.h, w.dt, w.mu, p)
    O.chi_update(sig, chi, D, sb, w.h, w.dt, p)
    b = O.div_rhs(ss, w.h, w.dt, w.mu)
    x = v.copy()
    O.wall_fill(x, w.h, O.BC(**w.bc_values()), t + w.dt)
    mg.vcycle(b, x)
    O.stress_final(x, ss, w.h, w.dt, w.lam, w.mu)


def rel_err(a, b):
    """(|a - b|_2 / |b|_2, max|a - b| / max|b|) of two tensors or arrays."""
    import torch
    if isinstance(a, torch.Tensor):
        d = a - b
        nb, mb = float(torch.linalg.vector_norm(b)), float(b.abs().max())
        return (float(torch.linalg.vector_norm(d)) / max(nb, 1e-300),
                float(d.abs().max()) / max(mb, 1e-300))
    d = a - b
    return (float(np.linalg.norm(d.ravel())) / max(float(np.linalg.norm(b.ravel())), 1e-300),
            float(np.abs(d).max()) / max(float(np.abs(b).max()), 1e-300))


# ------------------------------------------------------------------ ours

def lockstep(w, ctx_mixed, ctx64, v0, s0, c0, t0, nsteps, stream, dev):
    """Mixed and FP64 trajectories from the same initial state, one step of
    each in turn: per-step device times, cycles, and the mixed state's
    (norm-wise, element-wise) relative error against the FP64 state."""
    import torch

    from paper_1904_03808_gb300 import make_state
    st = {}
    for name in ("mixed", "fp64"):
        v, sg, c = (torch.from_numpy(a).to(dev) for a in (v0, s0, c0))
        st[name] = (v, sg, c, make_state(v, sg, c, t0))
    ctxs = {"mixed": ctx_mixed, "fp64": ctx64}
    ms = {"mixed": [], "fp64": []}
    cyc = {"mixed": 0, "fp64": 0}
    worst = 0.0
    err = {"v": [], "sigma": [], "chi": []}
    for _ in range(nsteps):
        for name in ("mixed", "fp64"):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, s = ctxs[name].step(st[name][3], w.dt, TOL)
            e1.record(stream)
            torch.cuda.synchronize()
            ms[name].append(e0.elapsed_time(e1))
            cyc[name] += s.cycles
            worst = max(worst, s.rel_resid)
        for i, key in ((0, "v"), (1, "sigma"), (2, "chi")):
            err[key].append(rel_err(st["mixed"][i], st["fp64"][i]))
    del st
    if nsteps == 0:
        return {"steps": 0}
    r3 = lambda x: float("%.3g" % x)  # noqa: E731
    return {"steps": nsteps, "from": "initial state (t0), both trajectories",
            "mixed_s_per_step": statistics.mean(ms["mixed"]) / 1e3,
            "fp64_s_per_step": statistics.mean(ms["fp64"]) / 1e3,
            "mixed_cycles_per_solve": cyc["mixed"] / nsteps,
            "fp64_cycles_per_solve": cyc["fp64"] / nsteps, "worst_rel_resid": worst,
            "max_err_v": max(e[1] for e in err["v"]) if nsteps else None,
            "max_err_sigma": max(e[1] for e in err["sigma"]) if nsteps else None,
            "max_err_chi": max(e[1] for e in err["chi"]) if nsteps else None,
            "err_v_per_step": [r3(e[1]) for e in err["v"]],
            "err_sigma_per_step": [r3(e[1]) for e in err["sigma"]],
            "err_note": "max|mixed - fp64| / max|fp64| after each step (element-wise); the "
                        "norm-wise errors are below these"}



def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1904_03808_gb300 as Q
    from paper_1904_03808_gb300 import MG_FP64, MG_MIXED, Context, binding, make_state

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    Q.lib()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    w = workload(args.n or 256)
    v0, s0, c0, t0 = w.initial_state()
    K = args.steps
    W = max(args.warmup, 3)

    def mk(prec):
        return Context(w.nx, w.ny, w.nz, w.h, I_K(), w.mu, bc=w.bc_values(), stz=w.stz,
                       precision=prec, max_cycles=100, inner_cycles=args.inner, stream=stream,
                       flags=binding.MG_FLAG_ADVECT_STRESS if args.advect else 0)

    vg = torch.from_numpy(v0).to(dev)
    sg = torch.from_numpy(s0).to(dev)
    cg = torch.from_numpy(c0).to(dev)
    state = make_state(vg, sg, cg, t0)
    ctx = mk(MG_MIXED)
    for _ in range(W):
        ctx.step(state, w.dt, TOL)
    # snapshot for the FP64 comparison and the oracle sample
    snap = (vg.clone(), sg.clone(), cg.clone(), state.t)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ctx.profile(True)
    clocks = Clocks(local)
    clocks.start()
    l0 = binding.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    # the K steps in one qs_run call (each step's stress correction fused
    # with the next step's predictor)
    _, run_stats = ctx.run(state, K, w.dt, TOL)
    ev1.record(stream)
    cyc = sum(s.cycles for s in run_stats)
    outer = sum(s.outer_iters for s in run_stats)
    worst = max(s.rel_resid for s in run_stats)
    torch.cuda.synchronize()
    launches = binding.launch_count() - l0
    clk = clocks.stop()
    t_step = max_over_ranks(ev0.elapsed_time(ev1) / 1e3 / K, ws, dev)
    if ws > 1:
        dist.barrier()
    sm_ms, sweeps, sm_launches = ctx.profile_read()
    ctx.profile(False)
    n_nodes = w.nx * w.ny * (w.nz - 1)
    t_sweep = sm_ms / 1e3 / max(sweeps, 1)
    achieved = SMOOTH_BYTES * n_nodes / t_sweep / 1e9
    peak, peak_kind = peak_hbm()
    traffic = traffic_per_sweep(n_nodes)

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    vh, sh, ch = (torch.from_numpy(a).pin_memory() for a in (v0, s0, c0))
    vh.copy_(snap[0])
    sh.copy_(snap[1])
    ch.copy_(snap[2])
    te = snap[3]
    Ke = max(2, min(K, 5))
    hstate = make_state(vg, sg, cg, te)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(Ke):
        vg.copy_(vh, non_blocking=True)
        sg.copy_(sh, non_blocking=True)
        cg.copy_(ch, non_blocking=True)
        ctx.step(hstate, w.dt, TOL)
        vh.copy_(vg, non_blocking=True)
        sh.copy_(sg, non_blocking=True)
        ch.copy_(cg, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3 / Ke, ws, dev)
    nbytes = (v0.nbytes + s0.nbytes + c0.nbytes)

    # ---- C3: mixed and FP64 in lockstep from the initial state, each step's
    # device time and the mixed state's error against the FP64 one
    ctx64 = mk(MG_FP64)
    lock = lockstep(w, ctx, ctx64, v0, s0, c0, t0, args.c3_steps, stream, dev)
    ctx.close()

    # ---- cold solve of a random right-hand side from v = 0 (mixed and FP64)
    from paper_1904_03808_gb300 import inputs as I
    bc = torch.from_numpy(I.rhs_field(1, w.nx, w.ny, w.nz)).to(dev)
    cold = {}
    for name, c in (("fp64", ctx64), ("mixed", mk(MG_MIXED))):
        x = torch.zeros_like(bc)
        x[0, 0], x[0, w.nz] = -1.0, 1.0
        c.solve(bc, x.clone(), TOL)  # warm-up of the code path
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        _, s = c.solve(bc, x, TOL)
        a1.record(stream)
        torch.cuda.synchronize()
        cold[name] = {"s": a0.elapsed_time(a1) / 1e3, "cycles": s.cycles,
                      "outer_iters": s.outer_iters, "rel_resid": s.rel_resid}
        if name == "mixed":
            c.close()
    del bc

    # ---- CPU oracle: one complete step from the timed steps' starting state
    # (rank 0, N = 1 only), beside one FP64 GPU step from the same state
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle as O
        vs, ss_, cs_ = (a.cpu().numpy() for a in snap[:3])
        mg = O.MG(w.nx, w.ny, w.nz, w.lam, w.mu)
        t_cpu, cyc_cpu = oracle_step(w, mg, vs, ss_, cs_, snap[3], advect=args.advect)
        mg.close()
        vg.copy_(snap[0])
        sg.copy_(snap[1])
        cg.copy_(snap[2])
        st64 = make_state(vg, sg, cg, snap[3])
        ctx64.step(st64, w.dt, TOL)
        ev, es = rel_err(vg.cpu().numpy(), vs), rel_err(sg.cpu().numpy(), ss_)
        cpu = {"value": t_cpu, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
               "sample": "one complete FP64 C oracle qs_step at %dx%dx%d (%d V-cycles to rel. "
                         "resid 1e-10), from the timed steps' starting state, timed end to end "
                         "(measured, not scaled)" % (w.nx, w.ny, w.nz, cyc_cpu),
               "gpu_fp64_vs_oracle": {"err_v": ev, "err_sigma": es,
                                      "note": "(norm-wise, element-wise) relative difference "
                                              "of the FP64 GPU step from the same state; two "
                                              "solves to 1e-10 differ by up to cond * 1e-10"}}
    ctx64.close()

    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": per_solve(t_step, ws), "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": W, "ms_per_step": t_step * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycles in f64 refinement",
        "data": "synthetic (seeded fields of the paper's recipes)",
        "config": config(w, {"precision": "mixed", "inner_cycles": args.inner,
                             "parallelism": "replicas" if ws > 1 else "single GPU",
                             **({"stress_advection": "ENO, MG_FLAG_ADVECT_STRESS"}
                                if args.advect else {})}),
        "solve": {"cycles_per_solve": cyc / K, "outer_per_solve": outer / K,
                  "worst_rel_resid": worst},
        "fp64": ({"value": lock["fp64_s_per_step"], "unit": UNIT, "steps": lock["steps"],
                  "cycles_per_solve": lock["fp64_cycles_per_solve"],
                  "speedup_mixed": lock["fp64_s_per_step"] / lock["mixed_s_per_step"],
                  "note": "mean over the C3 lockstep steps, mixed timed over the same steps"}
                 if lock["steps"] else None),
        "c3": lock,
        "cold_solve": cold,
        "roofline": {"bound": "hbm", "kernel": "finest-level FP32 Gauss-Seidel sweep",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes": SMOOTH_BYTES * n_nodes, "sweep_ms": t_sweep * 1e3,
                     "launches_per_sweep": sm_launches / max(sweeps, 1),
                     "share_of_step": sm_ms / 1e3 / K / t_step},
        "cpu_baseline": cpu,
        "e2e": {"value": per_solve(t_e2e, ws), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "steps": Ke},
        "gpu_launches": launches,
        "clocks": clk,
    }


def I_K():
    from paper_1904_03808_gb300 import inputs as I
    return I.TABLE1["K"]


# ------------------------------------------------------------- reference arm

def run_reference(args):
    """The FP64 CPU oracle as it stands, on this host's cores: each timed
    step is one complete oracle qs_step of the 256^3 workload (the oracle's
    own trajectory from the bench's initial state), timed end to end; each
    warm-up step a bounded pass over the step's arrays (pointwise pieces and
    one V-cycle) that leaves the state as it is.  Rank 0 only."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle as O
    O.build()
    w = workload(args.n or 256)
    v, sig, chi, t = w.initial_state()
    mg = O.MG(w.nx, w.ny, w.nz, w.lam, w.mu)
    for _ in range(args.warmup):
        oracle_touch(w, mg, v, sig, chi, t)
    secs, cycles = [], []
    for _ in range(args.steps):
        dt, cyc = oracle_step(w, mg, v, sig, chi, t)
        t += w.dt
        secs.append(dt)
        cycles.append(cyc)
    mg.close()
    value = float(np.mean(secs))
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "impl": "reference",
        "data": "synthetic (seeded fields of the paper's recipes)",
        "config": config(w, {"precision": "fp64 (CPU oracle)"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
                         "sample": "%d complete oracle qs_steps at %dx%dx%d (%.1f V-cycles a "
                                   "solve), each timed end to end (measured, not scaled); "
                                   "warm-up: the pointwise pieces and one V-cycle, %d times"
                                   % (args.steps, w.nx, w.ny, w.nz,
                                      float(np.mean(cycles)) if cycles else 0.0, args.warmup)},
        "per_step_s": [float("%.4g" % x) for x in secs],
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------------------ C2, CPU report, gradient

def run_c2(args):
    """128^3 cells, 100 FP64 steps of simple shear (strain 2% over the run):
    the GPU in lockstep with the CPU oracle, the GPU running the oracle's
    cycle count each step (tol 0), per-step (norm-wise, element-wise)
    relative difference of v, sigma and chi; both timed.  --preload sets the
    initial sigma_xz (default 1.2 GPa, the STZ-active variant; 0 is the
    literal unstressed start, elastic throughout)."""
    import torch

    import oracle as O
    from paper_1904_03808_gb300 import MG_FP64, Context, make_state
    from paper_1904_03808_gb300 import inputs as I
    n = args.n or 128
    K = args.steps
    pre = PRELOAD if args.preload is None else args.preload
    w = I.Workload(n, steps=K, strain=0.02, preload=pre, chi_mean=600.0, chi_std=30.0,
                   lc_cells=4.0, seed=2)
    v, sig, chi, t = w.initial_state()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    vg, sg, cg = (torch.from_numpy(a).to(dev) for a in (v, sig, chi))
    state = make_state(vg, sg, cg, t)
    mg = O.MG(w.nx, w.ny, w.nz, w.lam, w.mu)
    rows = []
    for k in range(K):
        t_cpu, cyc = oracle_step(w, mg, v, sig, chi, t)
        t += w.dt
        ctx = Context(w.nx, w.ny, w.nz, w.h, I.TABLE1["K"], w.mu, bc=w.bc_values(), stz=w.stz,
                      precision=MG_FP64, max_cycles=cyc, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, s = ctx.step(state, w.dt, 0.0)
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.close()
        row = {"step": k + 1, "cycles": cyc, "oracle_s": t_cpu, "gpu_ms": e0.elapsed_time(e1)}
        for key, a, b in (("v", vg, v), ("sigma", sg, sig), ("chi", cg, chi)):
            row["err_" + key] = rel_err(a.cpu().numpy(), b)
        rows.append(row)
    mg.close()
    worst = {key: max(max(r["err_" + key]) for r in rows) for key in ("v", "sigma", "chi")}
    return {"mode": "c2", "grid": [w.nx, w.ny, w.nz], "steps": K, "preload_pa": pre,
            "cores": O.threads(),
            "oracle_s_per_step": statistics.mean(r["oracle_s"] for r in rows),
            "oracle_s_total": sum(r["oracle_s"] for r in rows),
            "gpu_ms_per_step": statistics.mean(r["gpu_ms"] for r in rows[1:] or rows),
            "cycles_per_step": statistics.mean(r["cycles"] for r in rows),
            "worst_err": worst, "bar": 1e-12,
            "note": "GPU FP64 steps with the oracle's cycle count each step; err = max of "
                    "norm-wise and element-wise relative difference",
            "per_step": [{k: (float("%.3g" % x) if isinstance(x, float) else
                              [float("%.3g" % y) for y in x] if isinstance(x, tuple) else x)
                          for k, x in r.items()} for r in rows[::max(1, K // 20)]]}


def run_cpu_report(args):
    """The CPU oracle's complete runs (nothing scaled): a 32^3 single solve of
    a random right-hand side from v = 0, the 256^3 cold solve and the first 5
    steps of the bench workload, and the first step of the 512^3 disc
    workload."""
    import math

    import oracle as O
    from paper_1904_03808_gb300 import inputs as I
    out = {"mode": "cpu-report", "cores": O.threads()}
    try:
        out["cpu"] = [ln.split(":", 1)[1].strip() for ln in open("/proc/cpuinfo")
                      if ln.lower().startswith(("model name", "cpu part"))][:1]
    except OSError:
        pass

    def cold(n):
        b = I.rhs_field(1, n, n, n)
        x = np.zeros_like(b)
        x[0, 0], x[0, n] = -1.0, 1.0
        mg = O.MG(n, n, n, I.lame_lambda(I.TABLE1["K"], I.TABLE1["mu"]), I.TABLE1["mu"])
        t0 = time.perf_counter()
        st, cyc, _ = mg.solve(b, x, TOL, 100)
        dt = time.perf_counter() - t0
        mg.close()
        return {"s": dt, "cycles": cyc, "status": st}

    out["c1_32_cold_solve"] = cold(32)
    out["c3_256_cold_solve"] = cold(256)
    w = workload(256)
    v, sig, chi, t = w.initial_state()
    mg = O.MG(w.nx, w.ny, w.nz, w.lam, w.mu)
    steps = []
    for _ in range(5):
        dt, cyc = oracle_step(w, mg, v, sig, chi, t)
        t += w.dt
        steps.append({"s": dt, "cycles": cyc})
    mg.close()
    out["c3_256_first_5_steps"] = steps
    del v, sig, chi
    w5 = I.Workload(512, steps=20, kind=1, chi_mean=600.0, chi_std=30.0, lc_cells=8.0, seed=5,
                    dt_ts=2.0e3)
    w5.omega = 2.0 * math.pi / (1.0e8 * w5.ts)
    v, sig, chi, t = w5.initial_state()
    mg = O.MG(w5.nx, w5.ny, w5.nz, w5.lam, w5.mu)
    dt, cyc = oracle_step(w5, mg, v, sig, chi, t)
    mg.close()
    out["c5_512_first_step"] = {"s": dt, "cycles": cyc,
                                "workload": "disc kind 1, chi0 600 K / 30 K / l_c = 8 cells, "
                                            "dt = 2e3 t_s, from rest"}
    return out


def run_explicit(args):
    """The explicit method (section 3.2) against the quasi-static method on the
    comparison geometry of section 4: 64 x 64 x 32 cells (h = L/32, height L),
    simple shear, chi0 the cylindrical inclusion 600 K + 200 K
    exp(-500 (y^2 + z^2) / L^2) for |x| < L/2 (600 K elsewhere), sigma0 = 0,
    v0 = 0; the STZ time scale tau0 / zeta and wall speed 1e-7 zeta L / t_s;
    explicit steps dt_e <= t_s h^2 / (20 L^2) (the largest that divides the
    quasi-static step) with damping kappa = 4.8 (L / t_s) h; quasi-static steps
    of 100 t_s / zeta (mixed precision to 1e-10).  Reported: the explicit
    step's device time, and at intervals the root-mean-square differences
    (over cells, or corners for v) of chi, sigma and v between the two runs,
    normalised by chi_inf, s_Y and the wall speed."""
    import torch

    from paper_1904_03808_gb300 import MG_FP64, MG_MIXED, Context, make_state
    from paper_1904_03808_gb300 import inputs as I
    n, nz = 64, 32
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    out = {"mode": "explicit", "grid": [n, n, nz], "t_end_ts": args.t_end, "runs": []}
    for zeta in (float(z) for z in args.zeta.split(",")):
        w = I.Workload(n, steps=1, nz=nz, seed=1)
        L, h, ts = w.L, w.h, w.ts
        w.U_B = 1e-7 * zeta * L / ts
        stz = dict(w.stz)
        stz["tau0"] = stz["tau0"] / zeta
        x = -L + (np.arange(n) + 0.5) * h
        z = -0.5 * nz * h + (np.arange(nz) + 0.5) * h
        Z, Y, X = np.meshgrid(z, x, x, indexing="ij")
        chi0 = np.where(np.abs(X) < L / 2, 600.0 + 200.0 * np.exp(-500.0 * (Y * Y + Z * Z) / (L * L)),
                        600.0)
        v0 = np.zeros((3, nz + 1, n, n))
        s0 = np.zeros((6, nz, n, n))
        dt_qs = 100.0 * ts / zeta
        ne = int(math.ceil(dt_qs / (ts * h * h / (20.0 * L * L))))
        dt_e = dt_qs / ne
        kappa = 4.8 * L / ts * h
        runs = {}
        for name, prec in (("explicit", MG_FP64), ("qs", MG_MIXED)):
            ctx = Context(n, n, nz, h, I.TABLE1["K"], w.mu, bc=w.bc_values(), stz=stz,
                          precision=prec, max_cycles=100, stream=stream)
            ts_ = [torch.from_numpy(a.copy()).to(dev) for a in (v0, s0, chi0)]
            runs[name] = (ctx, ts_, make_state(*ts_, 0.0))
        nq = int(round(args.t_end * ts / dt_qs))
        every = max(1, nq // 20)
        rows, e_ms, q_ms = [], [], []
        for m in range(nq):
            for name in ("qs", "explicit"):
                ctx, _, st = runs[name]
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if name == "qs":
                    ctx.step(st, dt_qs, TOL)
                else:
                    ctx.explicit_step(st, dt_e, I.TABLE1["rho"], kappa, nsteps=ne)
                e1.record(stream)
                torch.cuda.synchronize()
                (q_ms if name == "qs" else e_ms).append(e0.elapsed_time(e1))
            if (m + 1) % every == 0 or m + 1 == nq:
                (vq, sq, cq), (ve, se, ce) = runs["qs"][1], runs["explicit"][1]
                rms = lambda d: float(torch.sqrt((d * d).sum(0).mean()))  # noqa: E731
                dsig = sq - se
                # Frobenius norm: off-diagonal components count twice
                fro = torch.sqrt((dsig[:3] ** 2).sum(0) + 2.0 * (dsig[3:] ** 2).sum(0))
                rows.append({"t_ts": float("%.4g" % ((m + 1) * dt_qs / ts)),
                             "chi": float("%.3g" % (rms((cq - ce)[None]) / w.stz["chi_inf"])),
                             "sigma": float("%.3g" % (float(torch.sqrt((fro * fro).mean())) /
                                                      w.stz["sY"])),
                             "v": float("%.3g" % (rms(vq - ve) / w.U_B)),
                             "chi_max_qs": float("%.4g" % float(cq.max()))})
        for ctx, _, _ in runs.values():
            ctx.close()
        out["runs"].append({"zeta": zeta, "dt_qs_ts": dt_qs / ts, "dt_e_ts": dt_e / ts,
                            "explicit_steps": ne * nq, "kappa_m2_s": kappa,
                            "explicit_ms_per_step": statistics.mean(e_ms[1:] or e_ms) / ne,
                            "qs_ms_per_step": statistics.mean(q_ms[1:] or q_ms),
                            "differences": rows})
    out["note"] = ("differences: root-mean-square over the grid of chi_qs - chi_e (/chi_inf), the "
                   "Frobenius norm of sigma_qs - sigma_e (/s_Y) and |v_qs - v_e| (/U_B)")
    return out


def run_grad(args):
    """The differentiation workload: 64^3 cells, 40 FP64 steps of simple
    shear from the STZ-active preload; the plastic work W alone
    (qs_plastic_work, no checkpoints) and W with dW/dchi0
    (qs_plastic_work_grad, checkpoints every --every steps), device times."""
    import torch

    from paper_1904_03808_gb300 import MG_FP64, MG_MIXED, Context, make_state
    from paper_1904_03808_gb300 import inputs as I
    n = args.n or 64
    K = args.steps if args.steps != 20 else 40
    w = I.Workload(n, steps=K, strain=0.02, preload=PRELOAD, chi_mean=600.0, chi_std=30.0,
                   lc_cells=4.0, seed=4)
    v, sig, chi, t = w.initial_state()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    out = {"mode": "grad", "grid": [w.nx, w.ny, w.nz], "steps": K, "checkpoint_every": args.every,
           "tol": TOL}
    for name, prec in (("fp64", MG_FP64), ("mixed", MG_MIXED)):
        ctx = Context(w.nx, w.ny, w.nz, w.h, I.TABLE1["K"], w.mu, bc=w.bc_values(), stz=w.stz,
                      precision=prec, max_cycles=100, stream=stream)
        res = {}
        for rep in range(2):  # the first round warms the code paths up
            for what in ("forward", "gradient"):
                vg, sg, cg = (torch.from_numpy(a).to(dev) for a in (v, sig, chi))
                state = make_state(vg, sg, cg, t)
                grad = torch.zeros_like(cg)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if what == "forward":
                    _, W, _ = ctx.plastic_work(state, K, w.dt, tol=TOL, checkpoint_every=K)
                else:
                    _, W, _ = ctx.plastic_work_grad(state, K, w.dt, grad, tol=TOL,
                                                    checkpoint_every=args.every)
                torch.cuda.synchronize()
                res[what] = {"s": time.perf_counter() - t0, "W": W}
                if what == "gradient":
                    res[what]["max_abs_grad"] = float(grad.abs().max())
        res["gradient_over_forward"] = res["gradient"]["s"] / res["forward"]["s"]
        out[name] = res
        ctx.close()
    out["note"] = ("host wall time of each call (each synchronises its stream); the gradient "
                   "call runs the forward steps with checkpoints, recomputes each segment and "
                   "runs the adjoint steps, each with one adjoint solve")
    return out


def run_fma_peak(args):
    """FP64 and FP32 fused multiply-add rates (csrc/peak_probe.cu, its own
    library), with the SM clocks sampled while they run."""
    import ctypes
    import torch
    from paper_1904_03808_gb300 import build as B
    B.build()
    torch.cuda.init()
    L = ctypes.CDLL(B.PROBE_LIB)
    L.qsmg_fma_peak.restype = ctypes.c_int
    L.qsmg_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    out = {"mode": "fma-peak", "kernel": "CTAs of 256 threads, 16 independent FMA chains a thread",
           "gpu": torch.cuda.get_device_name(0), "sms": torch.cuda.get_device_properties(0).multi_processor_count}
    for name, fp64, iters in (("fp64", 1, 20000), ("fp32", 0, 200000)):
        rows = []
        clocks = Clocks(0)
        clocks.start()
        for bpsm in (4, 8):
            tf, ms = ctypes.c_double(), ctypes.c_double()
            st = L.qsmg_fma_peak(fp64, bpsm, iters, 5, ctypes.byref(tf), ctypes.byref(ms))
            if st != 0:
                raise RuntimeError("qsmg_fma_peak failed with %d" % st)
            rows.append({"blocks_per_sm": bpsm, "tflops": tf.value, "ms": ms.value})
        out[name] = {"tflops": max(r["tflops"] for r in rows), "runs": rows,
                     "clocks": clocks.stop()}
    out["fp32_over_fp64"] = out["fp32"]["tflops"] / out["fp64"]["tflops"]
    return out


def main():
    args = parse()
    if args.sweep_only:
        out = run_sweeps(args)
    elif args.c2:
        out = run_c2(args)
    elif args.cpu_report:
        out = run_cpu_report(args)
    elif args.grad:
        out = run_grad(args)
    elif args.explicit:
        out = run_explicit(args)
    elif args.fma_peak:
        out = run_fma_peak(args)
    elif args.disc:
        out = run_disc(args)
    else:
        out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
