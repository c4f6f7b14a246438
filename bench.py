#!/usr/bin/env python3
"""Benchmark of the WENO-C finite-volume operator on one node.

A step is one SSP-RK3 time step (three stages of the whole hot path: time-step
reduction, cons->prim, WENO-W reconstruction, WENO-C limiter chain, Riemann
flux, conservative update), inputs resident in device memory.  The metric is
Mcell-updates/s per RK stage: interior cells x 3 stages / step time.

Headline (``value``): the learned-weight workload, 2-D circles and a planar
shock, 2048 x 2048 cells, N = 3 -- the one workload on which all three forms
of the metric exist: plain FP64 (``value``), the mixed precision and the
learned surrogate (``modes``), each with its L1 distance to the FP64 solution
after the same steps (matched accuracy).  ``configs`` carries the other
workloads with the same timing rules: the 1-D slab (a CUDA graph of 1,000
steps), the 1024 x 512 shock-bubble (N = 2), the 256^3 spheres and shock
(N = 3) and the 4,096 batched patches (graph replay, autotuned schedule),
each in FP64 and mixed precision with the L1 between them and the roofline
fraction of its sweeps.  Before the timed region the surrogate is trained on
the GPU from shock-bubble and 3-D states (``--no-learned`` skips the learned
lines); the scheme variants and the Phase-Field time step follow
(``--no-variants``).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle on this host's cores on the
headline workload (the oracle is the only other implementation of the
method).  Under torchrun each rank runs an independent replica of the
headline (the workload has no exchange step on one GPU per problem); value =
all cells updated / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-updates/s per RK stage"
WORKLOAD = ("circles_shock_2d {n}x{n} N=3 HLL CFL 0.2 outflow (64 circles, radii 10-80 "
            "cells, shock ratio 1e3, seeded): FP64 value, mixed and learned in modes")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n5", type=int, default=2048, help="edge of the headline circles grid")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the surrogate training and the learned-precision lines")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (slab, shock-bubble, 3-D, patches)")
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--train-batch", type=int, default=16384)
    ap.add_argument("--tau", type=float, default=1e-4)
    ap.add_argument("--n3d", type=int, default=256, help="edge of the 3-D workload")
    ap.add_argument("--steps3d", type=int, default=7, help="timed steps of the 3-D workload")
    ap.add_argument("--l1-steps2", type=int, default=200,
                    help="steps of the shock-bubble's mixed-vs-FP64 L1 run (its 200 RK3 steps)")
    ap.add_argument("--l1-steps3d", type=int, default=50,
                    help="steps of the 3-D workload's mixed-vs-FP64 L1 run (its 50 RK3 steps)")
    ap.add_argument("--npatch", type=int, default=4096)
    ap.add_argument("--steps4", type=int, default=6, help="timed steps of the patches")
    ap.add_argument("--n-adv", type=int, default=2048,
                    help="edge of the Sec. 4.1.1 advection grid that times the scheme variants")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the scheme variants (WENO-CL, WENO-W, WENO-JS, Kapila)")
    ap.add_argument("--profile", action="store_true",
                    help="only the timed steps of one precision on the headline workload "
                         "(a short run for profilers); prints the per-launch sweep time")
    ap.add_argument("--profile-3d", action="store_true",
                    help="as --profile on the 3-D spheres-and-shock workload (--n3d or "
                         "--profile-n cells a side)")
    ap.add_argument("--profile-precision", default="fp64", choices=["fp64", "mixed"],
                    help="precision of the --profile run")
    ap.add_argument("--profile-n", type=int, default=0,
                    help="edge of the --profile grid (0: the headline's)")
    ap.add_argument("--profile-pf", action="store_true",
                    help="only full time steps with the Phase-Field mechanism on the "
                         "shock-bubble (--steps of them after --warmup), for profilers")
    ap.add_argument("--profile-patches", action="store_true",
                    help="only --steps graph-replayed steps of the batched patches (--npatch "
                         "of them, --profile-precision, schedule kind --patch-kind), for "
                         "profilers")
    ap.add_argument("--patch-kind", type=int, default=2, choices=[0, 1, 2],
                    help="schedule kind of --profile-patches (0/1 persistent, 2 windows)")
    ap.add_argument("--profile-mlp", action="store_true",
                    help="only the surrogate kernels on the circles state (inference of one "
                         "direction, one training step of train_batch rows), for profilers")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_case(args, rank, n=None):
    from paper_2608_00746_b300 import inputs
    return inputs.circles_shock_2d(n=n or args.n5, seed=args.seed + rank)


def config_dict(args, ws):
    """The workload of both arms (identical dicts, so the two lines compare)."""
    state_mb = 9 * args.n5 * args.n5 * 8 / 1e6
    return {"workload": WORKLOAD.format(n=args.n5), "cells": args.n5 * args.n5, "nphase": 3,
            "dim": 2,
            "flux": "hll", "cfl": 0.2, "step": "one SSP-RK3 step (3 stages)",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
            "l2": f"state {state_mb:.0f} MB, larger than the 126 MB L2; the GPU arm also "
                  f"flushes L2 (256 MB write) between timed steps"}


# ---------------------------------------------------------------- reference arm
def oracle_step_rate(case, nsteps, warm=0, threads=0):
    """The FP64 CPU oracle as it stands, on this host's cores (threads > 0:
    that many)."""
    import oracle
    g = oracle.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                    bc=case.bc)
    all_threads = oracle.num_threads()
    if threads > 0:
        oracle.set_num_threads(threads)
    try:
        U = oracle.prim_to_cons(g, case.V)
        for _ in range(warm):
            U, _ = oracle.rk3_step(g, U, cfl=case.cfl)
        used = oracle.num_threads()
        t0 = time.perf_counter()
        for _ in range(nsteps):
            U, _ = oracle.rk3_step(g, U, cfl=case.cfl)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(all_threads)
    cells = int(np.prod(case.shape))
    return cells * 3 * nsteps / dt / 1e6, dt, used, U


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    case = make_case(args, 0)
    v, t, cores, _ = oracle_step_rate(case, args.steps, warm=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "Mcell/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args, ws),
        "cpu_baseline": {"value": round(v, 4), "unit": "Mcell/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"full grid, {args.steps} RK3 steps after {args.warmup}"},
        "e2e": {"value": round(v, 4), "unit": "Mcell/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"wenoc_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names[1:], start=5):
                if f[k].lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# the sources the FP64 window sweep (the roofline kernel) is built from
SWEEP_SOURCES = ("wenoc_device.cuh", "wenoc_sweep.cuh", "wenoc_window.cuh", "wenoc_fp64.cu")


def csrc_hash():
    """Hash of the roofline kernel's sources: a traffic record taken on other
    sources does not describe the kernel that runs."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2608_00746_b300", "csrc")
    for f in SWEEP_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel_hash, workload):
    """DRAM bytes per sweep launch of the roofline kernel on this workload from
    the committed ncu summary, when it was taken on the current kernel
    sources."""
    p = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("csrc_hash") != kernel_hash or d.get("workload") != workload:
        return None
    return d.get("dram_bytes_per_launch")


# ---------------------------------------------------------------- surrogate
def train_surrogate(args, dev):
    """Trains the weight surrogate on the GPU: feature rows and plain-weight
    targets of every face side of a 2-D shock-bubble state (1024 x 512, N = 2,
    third phase absent; initial and two later snapshots) and of a 3-D
    spheres-and-shock state (n3d^3, N = 3, after 25 steps), then
    train_steps Adam steps of train_batch rows, half from the rows whose
    plain weights differ from the ideal ones."""
    import torch
    from paper_2608_00746_b300 import inputs, surrogate, wenoc
    t0 = time.time()
    b = inputs.shock_bubble_2d(nx=1024, ny=512, seed=args.seed + 100)
    s3 = inputs.spheres_shock_3d(n=args.n3d, seed=args.seed + 200)
    rows = 3 * 2 * 2 * 1024 * 512 + 3 * 2 * args.n3d ** 3
    ts = surrogate.TrainingSet(rows, device=dev)
    for case, snaps, every in ((b, 3, 60), (s3, 1, 25)):
        g = wenoc.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                       bc=case.bc, precision="mixed")
        U = g.prim_to_cons(torch.from_numpy(case.V).to(dev))
        g.bind(U)
        for k in range(snaps):
            g.rk_step(cfl=case.cfl, nsteps=every if (k or case is s3) else 0)
            ts.add(g, U)
        g.sync_status()
        del g, U
    ts.finish()
    t1 = time.time()
    S = surrogate.Surrogate(seed=args.seed, device=dev)
    losses = S.train(ts, steps=args.train_steps, batch=args.train_batch, lr=3e-3,
                     lr_final=5e-5, seed=args.seed)
    t2 = time.time()
    info = {"rows": ts.nrows, "interesting_rows": ts.n_interesting,
            "samples": args.train_steps * args.train_batch,
            "loss_first": float(losses[:5].mean()), "loss_last": float(losses[-50:].mean()),
            "data_seconds": round(t1 - t0, 2), "train_seconds": round(t2 - t1, 2),
            "sources": "shock_bubble_2d 1024x512 (t0 + 2 snapshots), "
                       f"spheres_shock_3d {args.n3d}^3 (after 25 steps)"}
    del ts
    torch.cuda.empty_cache()
    return S, info


def group_l1(a, b, N, D):
    """max over variable groups (each mass, momentum vector, energy, each
    fraction) of the L1 distance relative to the reference's L1 norm."""
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    grps = [[p] for p in range(N)] + [list(range(N, N + D)), [N + D]] + \
        [[N + D + 1 + p] for p in range(N)]
    return max(((a[g] - b[g]).abs().sum() / a[g].abs().sum().clamp_min(1e-300)).item()
               for g in grps)


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as tdist
    from paper_2608_00746_b300 import replicas, roofline, wenoc

    ws, rank, local = dist_env()
    if ws > 1:
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if ws > 1:
            tdist.barrier()
        torch.cuda.synchronize()

    learned = not (args.no_learned or args.profile or args.profile_3d or args.profile_pf)
    S, train_info = train_surrogate(args, dev) if learned else (None, None)

    def make_grid(precision, c, counters=None, scheme="c", kmodel="allaire"):
        g = wenoc.Grid(c.shape, c.dx, c.gamma, c.pinf, c.D, flux=c.flux, bc=c.bc,
                       precision=precision, scheme=scheme, kmodel=kmodel)
        if precision == "learned":
            g.set_mlp(S.params, tau=args.tau, counters=counters)
        V = torch.from_numpy(c.V).to(dev)
        U = g.prim_to_cons(V)
        g.bind(U)
        return g, U

    # L2 flush buffer (larger than the 126 MB L2), written between timed steps
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def timed_steps(g, K, W, c, dt=0.0):
        """K timed RK steps (events per step, L2 flushed in between) and the
        mean duration of the sweep launches inside them (event pairs the
        library records around each direction's launches on the same
        stream: the sweep, preceded in learned precision by the surrogate).
        dt > 0: fixed time step, else from the CFL number on the device."""
        for _ in range(W):
            g.rk_step(cfl=c.cfl, dt=dt)
        barrier()
        s = torch.cuda.current_stream()
        evs = []
        g.sweep_timing_begin(K * 3 * c.dim)
        for _ in range(K):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            g.rk_step(cfl=c.cfl, dt=dt)
            e1.record(s)
            evs.append((e0, e1))
        barrier()
        nl, tot_sw, _ = g.sweep_timing_read()
        total = sum(e0.elapsed_time(e1) for e0, e1 in evs)
        g.sync_status()
        return total / K, tot_sw / max(nl, 1)  # ms per step, ms per sweep launch

    if args.profile_pf:
        from paper_2608_00746_b300 import inputs
        cb = inputs.shock_bubble_2d(nx=1024, ny=512, seed=args.seed)
        g, U = make_grid("fp64", cb)
        g.set_pf_workspace(U.device)
        g.step(cfl=cb.cfl, nsteps=args.warmup, tol=1e-12)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(cfl=cb.cfl, nsteps=args.steps, tol=1e-12)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / max(args.steps, 1)
        g.sync_status()
        it, rounds, res = g.pf_stats()
        band, per_thread = g.pf_band()
        print(json.dumps({"profile_pf": True, "ms_per_step": ms, "qmap_cg_iterations_last": it,
                          "qmap_unknowns_last": band, "qmap_unknowns_per_thread_last": per_thread,
                          "qmap_label_rounds_last": rounds, "qmap_residual_last": res,
                          "steps": args.steps, "warmup": args.warmup}), flush=True)
        return 0

    if args.profile or args.profile_3d:
        if args.profile_3d:
            from paper_2608_00746_b300 import inputs
            cp = inputs.spheres_shock_3d(n=args.profile_n or args.n3d, seed=args.seed)
        else:
            cp = make_case(args, 0, n=args.profile_n or None)
        g, U = make_grid(args.profile_precision, cp)
        ms, sw = timed_steps(g, args.steps, args.warmup, cp)
        print(json.dumps({"profile": True, "precision": args.profile_precision,
                          "cells": int(np.prod(cp.shape)), "ms_per_step": ms,
                          "sweep_ms_per_launch": sw, "steps": args.steps,
                          "warmup": args.warmup}), flush=True)
        return 0

    case = make_case(args, rank)
    N, D = case.N, case.dim
    cells = int(np.prod(case.shape))
    peak64 = roofline.PEAK_FP64_TFLOPS
    peak32 = roofline.PEAK_FP32_TFLOPS
    peak_bf16 = measured_bf16_peak()
    # FP64 DFMA probe of this GPU (context for the unit-count peak)
    peak_probe = wenoc.fp64_peak() / 1e12

    modes = ("fp64", "mixed", "learned") if learned else ("fp64", "mixed")
    results = {}
    configs = {}
    infer = None
    with Clocks(local) as clk:
        time.sleep(1.0)  # let the sampler start before the timed region
        for prec in modes:
            g, U = make_grid(prec, case)
            results[prec] = timed_steps(g, args.steps, args.warmup, case)
            del g, U
        if learned and rank == 0:
            infer = time_inference(case, S, make_grid, barrier, dev)
        if rank == 0 and not args.no_configs:
            configs = run_configs(args, make_grid, timed_steps, barrier, dev, learned)
        variants = run_variants(args, rank, make_grid, timed_steps)
    clocks = clk.summary()

    def matched_l1(c, K):
        """Reduced modes against FP64 after K steps from the same initial
        state with the same time steps: group L1 and, for the learned mode,
        the share of non-flat face sides that took the surrogate's weights."""
        g64, U64 = make_grid("fp64", c)
        others = {}
        cnt = torch.zeros(2, dtype=torch.int64, device=dev)
        for prec in modes[1:]:
            others[prec] = make_grid(prec, c, counters=cnt if prec == "learned" else None)
        for _ in range(K):
            dt = g64.rk_step(cfl=c.cfl, want_dt=True)
            for g, _ in others.values():
                g.rk_step(dt=dt)
        out = {prec: group_l1(U64, U, c.N, c.dim) for prec, (g, U) in others.items()}
        dec, fb = cnt.tolist()
        acc = (1.0 - fb / dec) if dec else None
        for g, _ in others.values():
            g.sync_status()
        del g64, U64, others
        return out, acc

    l1s, acc = matched_l1(case, args.steps)

    # end to end through the C ABI with host buffers (wc_rk_step_host: the
    # upload overlaps the first sweep, the download the last one)
    g, U = make_grid("fp64", case)
    host = torch.empty(U.numel(), dtype=torch.float64, pin_memory=True)
    host.copy_(U.reshape(-1).cpu())
    nbytes = U.numel() * 8
    for _ in range(args.warmup):  # (the first call creates the copy stream and its events)
        g.rk_step_host(host, cfl=case.cfl)
    torch.cuda.synchronize()
    barrier()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        g.rk_step_host(host, cfl=case.cfl)
    e1.record(s)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    del g, U, host

    ms = {prec: results[prec][0] for prec in modes}
    sw = {prec: results[prec][1] for prec in modes}
    # max over ranks (replicas: the job takes as long as the slowest rank)
    vals = replicas.max_over_ranks([ms[p] for p in modes] + [e2e_ms], device=dev)
    ms = dict(zip(modes, vals[:len(modes)]))
    e2e_ms = vals[len(modes)]
    value = replicas.weak_value(ws, cells, 3, ms["fp64"])
    e2e = replicas.weak_value(ws, cells, 3, e2e_ms)

    fl = roofline.flops_per_cell_dir(N, D, "hll")
    achieved = fl * cells / (sw["fp64"] * 1e-3) / 1e12
    khash = csrc_hash()
    traffic = traffic_from_profile(khash, f"circles_shock_2d {args.n5}x{args.n5}")
    mode_lines = {"fp64": {"value": round(value, 3), "ms_per_step": round(ms["fp64"], 4),
                           "ms_per_direction": round(sw["fp64"], 4)}}
    rl_modes = {}
    for prec in modes[1:]:
        v = replicas.weak_value(ws, cells, 3, ms[prec])
        mode_lines[prec] = {"value": round(v, 3), "ms_per_step": round(ms[prec], 4),
                            "ms_per_direction": round(sw[prec], 4),
                            "speedup_vs_fp64": round(ms["fp64"] / ms[prec], 3),
                            "l1_rel_vs_fp64_max_var": l1s[prec], "l1_steps": args.steps}
        rl_modes[prec] = mode_roofline(N, D, cells, sw[prec], peak64, peak32, peak_bf16,
                                       learned=prec == "learned")
    if learned:
        mode_lines["learned"].update({"tau": args.tau, "accepted_face_sides": acc})
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Mcell/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms["fp64"], 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded circles-and-shock initial condition)",
        "config": config_dict(args, ws),
        "modes": mode_lines,
        "roofline": {
            "bound": "alu", "kernel": "k_sweep_win<N=3,D=2,double> (window direction sweep)",
            "achieved": round(achieved, 4), "peak": round(peak64, 4), "unit": "TFLOP/s",
            "frac": round(achieved / peak64, 4), "traffic": traffic,
            "peak_source": "unit count x clock: 2 DFMA/clk/SM x 2 flop x 148 SM x 2032 MHz "
                           "(MEASURED_PEAKS.json has no FP64 figure)",
            "peak_probe_measured": round(peak_probe, 4),
            "flops_per_cell_dir": fl, "flops_source": "oracle op counter (op_counts.json)",
            "sweep_ms_per_launch": round(sw["fp64"], 4),
            "hbm_bytes_per_cell_stage_min": roofline.bytes_per_cell_stage(N, D),
            "modes": rl_modes,
        },
        "clocks": clocks,
        "e2e": {"value": round(e2e, 3), "unit": "Mcell/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        # a step: per stage the primitive-slot pass (the first one also takes
        # the CFL rate) and D sweeps
        "gpu_launches": args.steps * 3 * (1 + D),
        "csrc_hash": khash,
    }
    if learned:
        line["surrogate_training"] = train_info
    if infer:
        line["surrogate_inference"] = infer
    if configs:
        line["configs"] = configs
    if variants:
        line["scheme_variants"] = variants
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baselines(args, case)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        tdist.destroy_process_group()
    return 0


def measured_bf16_peak():
    """Dense BF16 peak (TFLOP/s) from MEASURED_PEAKS.json when present (the
    burst figure: the inference is timed alone), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"])
    except Exception:
        return 1800.0


def mode_roofline(N, D, cells, ms_dir, peak64, peak32, peak_bf16, learned=False):
    """Roofline of one direction of the reduced-precision forms: the FP64 and
    FP32 flops of the oracle's count split as the mixed form assigns them,
    each at its pipe's peak, plus (learned) the surrogate's BF16 contraction
    of both face sides at the measured BF16 peak; the bound is the slowest
    of those times, and frac = bound time / measured time per direction."""
    from paper_2608_00746_b300 import roofline
    f64, f32 = roofline.mixed_split(N, D, "hll")
    t64 = f64 * cells / (peak64 * 1e12)
    t32 = f32 * cells / (peak32 * 1e12)
    ttc = 2 * roofline.MLP_FLOPS_PER_FACE_SIDE * cells / (peak_bf16 * 1e12) if learned else 0.0
    t = max(t64, t32, ttc)
    bound = "alu (fp64)" if t == t64 else ("alu (fp32)" if t == t32 else "tensor (bf16)")
    return {"bound": bound, "fp64_flops_per_cell_dir": f64, "fp32_flops_per_cell_dir": f32,
            "tensor_flops_per_cell_dir": 2 * roofline.MLP_FLOPS_PER_FACE_SIDE if learned else 0,
            "t_fp64_ms": round(t64 * 1e3, 4), "t_fp32_ms": round(t32 * 1e3, 4),
            "t_tensor_ms": round(ttc * 1e3, 4), "ms_per_direction": round(ms_dir, 4),
            "frac": round(t * 1e3 / ms_dir, 4),
            "peaks_tflops": {"fp64": round(peak64, 3), "fp32": round(peak32, 3),
                             "bf16_measured": peak_bf16}}


def time_inference(case, S, make_grid, barrier, dev):
    """The surrogate's inference kernel alone, one direction of the headline."""
    import torch
    from paper_2608_00746_b300 import roofline
    g, U = make_grid("mixed", case)
    W5 = torch.empty((18, g.ncell), dtype=torch.float32, device=dev)
    st5 = torch.zeros(1, dtype=torch.int32, device=dev)
    for _ in range(3):
        g.mlp_infer(U, 0, S.params, W5, st5)
    barrier()
    s_ = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_)
    for _ in range(10):
        g.mlp_infer(U, 0, S.params, W5, st5)
    e1.record(s_)
    barrier()
    ms = e0.elapsed_time(e1) / 10
    rows = 2 * g.ncell
    fl_row = roofline.MLP_FLOPS_PER_FACE_SIDE
    tf = fl_row * rows / (ms * 1e-3) / 1e12
    peak = measured_bf16_peak()
    return {"kernel": "k_mlp_infer2<3,2> (stencil gather, features of both face sides, 4 tcgen05 layers)",
            "rows": rows, "ms_per_launch": round(ms, 4), "achieved_tflops": round(tf, 2),
            "flops_per_row": fl_row, "frac_of_bf16_measured": round(tf / peak, 4)}


def run_configs(args, make_grid, timed_steps, barrier, dev, learned):
    """The other workloads, FP64 and mixed precision (and learned on the
    shock-bubble), each with the L1 of mixed against FP64 after the timed
    steps' count and the roofline fraction of its FP64 sweeps."""
    import torch
    from paper_2608_00746_b300 import inputs, roofline, wenoc
    peak64 = roofline.PEAK_FP64_TFLOPS
    out = {}

    def line(c, res, K, flux="hll", extra=None):
        cells = int(np.prod(c.shape))
        N, D = c.N, c.dim
        d = {}
        for prec, (ms, sw) in res.items():
            d[prec] = {"value": round(cells * 3 / (ms * 1e-3) / 1e6, 3),
                       "ms_per_step": round(ms, 4), "ms_per_direction": round(sw, 4)}
        fl = roofline.flops_per_cell_dir(N, D, flux)
        d["fp64"]["frac"] = round(fl * cells / (res["fp64"][1] * 1e-3) / 1e12 / peak64, 4)
        d["mixed"]["speedup_vs_fp64"] = round(res["fp64"][0] / res["mixed"][0], 3)
        if extra:
            d.update(extra)
        d["steps"] = K
        return d

    def l1_pair(c, K, flux_dt=None):
        g64, U64 = make_grid("fp64", c)
        gm, Um = make_grid("mixed", c)
        for _ in range(K):
            dt = g64.rk_step(cfl=c.cfl, dt=flux_dt or 0.0, want_dt=True)
            gm.rk_step(dt=dt)
        gm.sync_status()
        g64.sync_status()
        return group_l1(U64, Um, c.N, c.dim)

    # config 2: 2-D shock-bubble 1024 x 512, N = 2 (all three forms)
    c2 = inputs.shock_bubble_2d(nx=1024, ny=512, seed=args.seed)
    res = {}
    for prec in (("fp64", "mixed", "learned") if learned else ("fp64", "mixed")):
        g, U = make_grid(prec, c2)
        res[prec] = timed_steps(g, args.steps, 3, c2)
        del g, U
    d2 = line(c2, res, args.steps)
    d2["mixed"]["l1_rel_vs_fp64_max_var"] = l1_pair(c2, args.l1_steps2)
    d2["mixed"]["l1_after_steps"] = args.l1_steps2
    if learned:
        d2["learned"]["speedup_vs_fp64"] = round(res["fp64"][0] / res["learned"][0], 3)
    out["shock_bubble_2d"] = dict(workload="shock_bubble_2d 1024x512 N=2 HLL CFL 0.2 "
                                  "reflective (seeded)", **d2)

    # config 3: 3-D spheres and shock, 256^3, N = 3
    c3 = inputs.spheres_shock_3d(n=args.n3d, seed=args.seed)
    res = {}
    for prec in ("fp64", "mixed"):
        g, U = make_grid(prec, c3)
        res[prec] = timed_steps(g, args.steps3d, 2, c3)
        del g, U
        torch.cuda.empty_cache()
    d3 = line(c3, res, args.steps3d)
    d3["mixed"]["l1_rel_vs_fp64_max_var"] = l1_pair(c3, args.l1_steps3d)
    d3["mixed"]["l1_after_steps"] = args.l1_steps3d
    out["spheres_shock_3d"] = dict(workload=f"spheres_shock_3d {args.n3d}^3 N=3 HLL CFL 0.2 "
                                   "outflow (16 spheres, shock ratio 1e3, seeded)", **d3)
    del c3
    torch.cuda.empty_cache()

    # config 1: the 1-D slab, a CUDA graph of 1,000 steps replayed
    c1 = inputs.interface_advection_1d(n=200)
    res = {}
    states = {}
    for prec in ("fp64", "mixed"):
        g, U = make_grid(prec, c1)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            dt1 = g.rk_step(cfl=c1.cfl, nsteps=1, want_dt=True)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=st):
            g.rk_step(dt=dt1, nsteps=1000)
        graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        g.sync_status()
        ms = e0.elapsed_time(e1) / 1000
        res[prec] = (ms, ms / 3)
        states[prec] = U
    d1 = line(c1, res, 2001, flux="hllc")
    d1["mixed"]["l1_rel_vs_fp64_max_var"] = group_l1(states["fp64"], states["mixed"], 2, 1)
    V = {p: g.cons_to_prim(states[p]).cpu().numpy() for p in states}
    d1["equilibrium_after_2001_steps"] = {
        p: {"u_dev_max": float(np.abs(V[p][2] - 1.0).max()),
            "P_dev_max_of_scale": float(np.abs(V[p][3] - 1e5).max() / (1e5 + 6e8))}
        for p in V}
    out["interface_advection_1d"] = dict(
        workload="interface_advection_1d 200 cells N=2 HLLC CFL 0.5 periodic (CUDA graph "
                 "of 1000 steps; latency-bound)", **d1)

    # config 4: 4,096 batched patches, graph replay, autotuned schedule
    from paper_2608_00746_b300 import autotune
    edges, pstates, (gm_, pi_, Dm_) = inputs.patch_batch(npatch=args.npatch, seed=args.seed)
    res = {}
    finals = {}
    sched = {}
    for prec in ("fp64", "mixed"):
        P = wenoc.Patches(edges, gm_, pi_, Dm_, precision=prec)
        V4 = torch.from_numpy(P.pack(pstates)).to(dev)
        U4 = P.prim_to_cons(V4)
        del V4
        P.bind(U4)
        U_init = U4.clone()
        sched[prec] = autotune.tuned_schedule(P, 0.2, prec, "hll", 3, steps=2)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            P.rk_step(cfl=0.2, nsteps=1, use_graph=True)   # captures the step graph
        torch.cuda.synchronize()
        U4.copy_(U_init)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            P.rk_step(cfl=0.2, nsteps=args.steps4, use_graph=True)
            e1.record(st)
        torch.cuda.synchronize()
        P.sync_status()
        ms = e0.elapsed_time(e1) / args.steps4
        res[prec] = (ms, ms / 3)
        finals[prec] = U4
        del U_init, P
    ncell4 = finals["fp64"].shape[1]
    fl = roofline.flops_per_cell_dir(3, 3, "hll")
    d4 = {}
    for prec, (ms, _) in res.items():
        kind = {0: "persistent, static", 1: "persistent, queue", 2: "window sweeps"}
        d4[prec] = {"value": round(ncell4 * 3 / (ms * 1e-3) / 1e6, 3), "ms_per_step": round(ms, 4),
                    "schedule": dict(sched[prec], kind=kind.get(sched[prec]["dynamic"]))}
    d4["fp64"]["frac"] = round(fl * 3 * ncell4 * 3 / (res["fp64"][0] * 1e-3) / 1e12 / peak64, 4)
    d4["mixed"]["speedup_vs_fp64"] = round(res["fp64"][0] / res["mixed"][0], 3)
    d4["mixed"]["l1_rel_vs_fp64_max_var"] = group_l1(finals["fp64"], finals["mixed"], 3, 3)
    d4["steps"] = args.steps4
    d4["cells"] = int(ncell4)
    out["patches"] = dict(workload=f"patch_batch {args.npatch} cube patches, edges "
                          "{8,12,16,24,32}, N=3 HLL CFL 0.2 (dt on the device each step), "
                          "autotuned schedule (one persistent launch per stage, or window "
                          "sweeps per group of equal patches), CUDA graph replay; L1 of mixed "
                          "against FP64 after the timed steps", **d4)
    del finals
    torch.cuda.empty_cache()
    return out


def cpu_baselines(args, case):
    """The FP64 oracle as it stands on this host: all cores on one RK3 step of
    the headline grid, and one thread on one step of a 512 x 512 instance of
    the same workload generator (seeded alike)."""
    out = {}
    try:
        v, t, cores, _ = oracle_step_rate(case, 1)
        out = {"value": round(v, 4), "unit": "Mcell/s", "cores": cores, "kind": "oracle",
               "sample": f"one RK3 step of the full {args.n5}x{args.n5} grid ({t:.1f} s)"}
        small = make_case(args, 0, n=512)
        v1, t1, c1, _ = oracle_step_rate(small, 1, threads=1)
        out["single_thread"] = {"value": round(v1, 4), "unit": "Mcell/s", "cores": c1,
                                "sample": f"one RK3 step of a 512x512 circles-and-shock grid "
                                          f"({t1:.1f} s)"}
    except Exception as e:  # the oracle must be built on the host
        out = {"value": None, "error": str(e)[:200]}
    return out


def run_variants(args, rank, make_grid, timed_steps):
    """The scheme variants, each on its own workload, FP64, same timing as the
    headline: WENO-C, WENO-CL and the WENO-W / WENO-JS comparison schemes on
    the Sec. 4.1.1 air-circle advection (n^2, dt = 0.1 n^-1, the paper's
    1e-3 at n = 100) with the consistency error after the run; the Kapila
    model and the full time step with the Phase-Field mechanism on the
    1024 x 512 shock-bubble."""
    if args.no_variants or rank != 0:
        return None
    from paper_2608_00746_b300 import inputs
    out = {}
    cA = inputs.two_phase_advection_2d(n=args.n_adv)
    dtA = 0.1 / args.n_adv
    cells = args.n_adv ** 2
    rho1 = cA.meta["rho"][0]
    adv = {"workload": f"two_phase_advection_2d {args.n_adv}x{args.n_adv} N=2 HLLC periodic "
                       f"dt {dtA:.3g} (Sec. 4.1.1 layout)", "steps": args.steps}
    for scheme in ("c", "cl", "w", "js"):
        g, U = make_grid("fp64", cA, scheme=scheme)
        ms, sw = timed_steps(g, args.steps, 3, cA, dt=dtA)
        cons = (U[0] / rho1 - U[5]).abs().max().item()
        # Eq. 29 with the Sec. 4.1.1 heat capacities (T = 300 at P0 = 4.819e-5)
        A = [1.0 / (gm - 1.0) for gm in cA.gamma]
        cT = [(A[p] * 4.819e-5 + cA.gamma[p] * cA.pinf[p] * A[p] - cA.pinf[p])
              / (cA.meta["rho"][p] * 300.0) for p in range(2)]
        temp = (g.temperature(U, cT) / 300.0 - 1.0).abs().max().item()
        adv[scheme] = {"value": round(cells * 3 / (ms * 1e-3) / 1e6, 3),
                       "ms_per_step": round(ms, 4), "ms_per_direction": round(sw, 4),
                       "consistency_error_max": cons, "temperature_error_max": temp}
        del g, U
    out["advection"] = adv
    cb = inputs.shock_bubble_2d(nx=1024, ny=512, seed=args.seed)
    g, U = make_grid("fp64", cb, kmodel="kapila")
    ms, sw = timed_steps(g, args.steps, 3, cb)
    cells_h = int(np.prod(g.shape))
    out["kapila"] = {"workload": "shock_bubble_2d 1024x512, K_p of the Kapila model",
                     "value": round(cells_h * 3 / (ms * 1e-3) / 1e6, 3),
                     "ms_per_step": round(ms, 4), "ms_per_direction": round(sw, 4)}
    del g, U
    out["phase_field"] = time_phase_field(make_grid, cb)
    return out


def time_phase_field(make_grid, cb, K=20):
    """Full time steps of Sec. 2.2 on the 1024 x 512 shock-bubble: the
    hyperbolic step, Eq. 28, the Q-map of Eq. 4 (conjugate gradients to a
    D-weighted residual of 1e-12, started from the previous step's Q) and
    the Phase-Field step, FP64; then each part timed alone."""
    import torch
    g, U = make_grid("fp64", cb)
    g.set_pf_workspace(U.device)
    g.step(cfl=0.2, nsteps=3, tol=1e-12)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    g.step(cfl=0.2, nsteps=K, tol=1e-12)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    iters, rounds, res = g.pf_stats()
    band, per_thread = g.pf_band()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    parts = np.zeros(4)
    Q = None
    for _ in range(5):
        ev[0].record(s)
        dt = g.rk_step(cfl=0.2, want_dt=True)
        ev[1].record(s)
        g.cac_rhs(U)
        ev[2].record(s)
        Q, _, _ = g.qmap(U, Q=Q, tol=1e-12, warm=Q is not None)
        ev[3].record(s)
        g.pf_step(Q, dt)
        ev[4].record(s)
        torch.cuda.synchronize()
        parts += [ev[k].elapsed_time(ev[k + 1]) for k in range(4)]
    g.sync_status()
    parts /= 5
    cells = int(np.prod(g.shape))
    del g, U
    mixed = time_phase_field_mixed(make_grid, cb, K)
    return {"workload": "shock_bubble_2d 1024x512, full time step (hyperbolic + Eq. 28 + "
                        "Eq. 4 + Phase-Field step), Q-map tolerance 1e-12",
            "mixed": mixed,
            "steps": K, "value": round(cells * 3 / (ms * 1e-3) / 1e6, 3), "unit": "Mcell/s",
            "ms_per_step": round(ms, 4), "qmap_cg_iterations_last": iters,
            "qmap_label_rounds_last": rounds, "qmap_residual_last": res,
            "qmap_unknowns_last": band, "qmap_unknowns_per_thread_last": per_thread,
            "ms_hyperbolic": round(parts[0], 4), "ms_eq28": round(parts[1], 4),
            "ms_qmap": round(parts[2], 4), "ms_pf_step": round(parts[3], 4)}


def time_phase_field_mixed(make_grid, cb, K):
    """The same full time steps in the mixed precision (the sweeps of both
    steps in the split mixed form, the Q-map in FP64): K steps at the fixed
    time step of the FP64 grid's first CFL step, timed after 3 warm-up steps
    from the same state, and the L1 distance to K FP64 steps at that time
    step (matched accuracy)."""
    import torch
    g64, U64 = make_grid("fp64", cb)
    g64.set_pf_workspace(U64.device)
    gm, Um = make_grid("mixed", cb)
    gm.set_pf_workspace(Um.device)
    U0 = U64.clone()
    dt = g64.step(cfl=0.2, nsteps=1, tol=1e-12, want_dt=True)
    U64.copy_(U0)
    g64.set_pf_workspace(U64.device)  # a fresh Q-map start
    gm.step(dt=dt, nsteps=3, tol=1e-12)
    Um.copy_(U0)
    gm.set_pf_workspace(Um.device)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    gm.step(dt=dt, nsteps=K, tol=1e-12)
    e1.record(s)
    g64.step(dt=dt, nsteps=K, tol=1e-12)
    torch.cuda.synchronize()
    gm.sync_status()
    g64.sync_status()
    ms = e0.elapsed_time(e1) / K
    cells = int(np.prod(gm.shape))
    l1 = group_l1(U64, Um, cb.N, cb.dim)
    del g64, U64, gm, Um, U0
    return {"steps": K, "dt": dt, "value": round(cells * 3 / (ms * 1e-3) / 1e6, 3),
            "unit": "Mcell/s", "ms_per_step": round(ms, 4), "l1_rel_vs_fp64_max_var": l1}


def run_profile_patches(args):
    """The batched patches alone: --warmup then --steps steps (CFL 0.2, direct
    launches: the kernels of the graph-replayed benchmark step) in one
    precision and schedule kind (128-thread blocks, 2 per SM persistent or 4
    per SM in windows), events around the timed steps."""
    import torch
    from paper_2608_00746_b300 import inputs, wenoc
    dev = torch.device("cuda", 0)
    edges, states, (gm, pi, Dm) = inputs.patch_batch(npatch=args.npatch, seed=args.seed)
    P = wenoc.Patches(edges, gm, pi, Dm, precision=args.profile_precision)
    V = torch.from_numpy(P.pack(states)).to(dev)
    U = P.prim_to_cons(V)
    del V
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        P.bind(U, stream=s)
        P.set_schedule(128, 4 if args.patch_kind == 2 else 2, args.patch_kind)
        P.rk_step(cfl=0.2, nsteps=max(args.warmup, 1), stream=s)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        P.rk_step(cfl=0.2, nsteps=args.steps, stream=s)
        e1.record(s)
    s.synchronize()
    P.sync_status(stream=s)
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    print(json.dumps({"profile_patches": True, "precision": args.profile_precision,
                      "kind": args.patch_kind, "npatch": args.npatch, "cells": int(P.ncell),
                      "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup}), flush=True)
    return 0


def run_profile_mlp(args):
    """Surrogate kernels alone (untrained network: the timing does not depend
    on the weights): 3 + 5 inference launches of direction 0 of the circles
    state and one training step, events around each group."""
    import torch
    from paper_2608_00746_b300 import inputs, surrogate, wenoc
    dev = torch.device("cuda", 0)
    c5 = inputs.circles_shock_2d(n=args.n5, seed=args.seed)
    g = wenoc.Grid(c5.shape, c5.dx, c5.gamma, c5.pinf, c5.D, flux=c5.flux, bc=c5.bc,
                   precision="mixed")
    U = g.prim_to_cons(torch.from_numpy(c5.V).to(dev))
    g.bind(U)
    S = surrogate.Surrogate(seed=args.seed, device=dev)
    W = torch.empty((18, g.ncell), dtype=torch.float32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    for _ in range(3):
        g.mlp_infer(U, 0, S.params, W, st)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    for _ in range(5):
        g.mlp_infer(U, 0, S.params, W, st)
    e[1].record()
    ts = surrogate.TrainingSet(2 * g.ncell, device=dev)
    ts.add(g, U, directions=[0])
    ts.finish()
    idx = torch.randint(0, ts.nrows, (args.train_batch,), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    e[2].record()
    S.train_step(ts.X, ts.T, idx, 1e-3)
    e[3].record()
    torch.cuda.synchronize()
    S.check_status()
    rows = 2 * g.ncell
    infer_ms = e[0].elapsed_time(e[1]) / 5
    print(json.dumps({"profile_mlp": True, "rows": rows, "infer_ms": infer_ms,
                      "infer_tflops": 21376 * rows / (infer_ms * 1e-3) / 1e12,
                      "train_step_ms": e[2].elapsed_time(e[3]), "batch": args.train_batch}),
          flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_mlp:
        return run_profile_mlp(args)
    if args.profile_patches:
        return run_profile_patches(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
