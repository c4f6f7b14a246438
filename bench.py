#!/usr/bin/env python3
"""Benchmark of the WENO-C finite-volume operator on one node.

A step is one SSP-RK3 time step (three stages of the whole hot path: time-step
reduction, cons->prim, WENO-W reconstruction, WENO-C limiter chain, Riemann
flux, conservative update) on the 2-D two-phase shock-bubble workload,
1024 x 512 cells, N = 2 (air bubble in water hit by a planar shock, seeded),
inputs resident in device memory.  The metric is Mcell-updates/s per RK stage:
interior cells x 3 stages / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Beside the FP64 headline the line carries the mixed and learned precisions
on the same workload (speed and group L1 against FP64 after the same steps),
the learned-weight workload (2-D circles and shock, 2048 x 2048, N = 3) in all
three precisions, and the surrogate's training record: before the timed
region the surrogate is trained on the GPU from shock-bubble and 3-D
spheres-and-shock states (``--no-learned`` skips all of this).  The scheme
variants follow (``--no-variants`` skips them): WENO-C, WENO-CL and the
WENO-W / WENO-JS comparison schemes on the Sec. 4.1.1 advection, the Kapila
model, and the full time step with the Phase-Field mechanism (Eq. 28, the
Q-map of Eq. 4, the Phase-Field step) on the headline workload.

``--impl reference`` times the FP64 CPU oracle on this host's cores on the same
workload (the oracle is the only other implementation of the method).
Under torchrun each rank runs an independent replica (the workload has no
exchange step on one GPU per problem); value = all cells updated / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-updates/s per RK stage"
WORKLOAD = "shock_bubble_2d 1024x512 N=2 HLL CFL 0.2 reflective (seeded)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=512)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the surrogate training and the learned-precision lines")
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--train-batch", type=int, default=16384)
    ap.add_argument("--tau", type=float, default=1e-4)
    ap.add_argument("--n3d", type=int, default=256, help="edge of the 3-D training source")
    ap.add_argument("--n5", type=int, default=2048, help="edge of the 2-D circles workload")
    ap.add_argument("--steps5", type=int, default=20)
    ap.add_argument("--n-adv", type=int, default=2048,
                    help="edge of the Sec. 4.1.1 advection grid that times the scheme variants")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the scheme variants (WENO-CL, WENO-W, WENO-JS, Kapila)")
    ap.add_argument("--profile", action="store_true",
                    help="only the timed steps of one precision (a short run for profilers); "
                         "prints the per-launch sweep time")
    ap.add_argument("--profile-precision", default="fp64", choices=["fp64", "mixed"],
                    help="precision of the --profile run")
    ap.add_argument("--profile-pf", action="store_true",
                    help="only full time steps with the Phase-Field mechanism on the headline "
                         "workload (--steps of them after --warmup), for profilers")
    ap.add_argument("--profile-mlp", action="store_true",
                    help="only the surrogate kernels on the circles state (inference of one "
                         "direction, one training step of train_batch rows), for profilers")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_case(args, rank):
    from paper_2608_00746_b300 import inputs
    return inputs.shock_bubble_2d(nx=args.nx, ny=args.ny, seed=args.seed + rank)


def config_dict(args, ws, flush):
    return {"workload": WORKLOAD, "cells": args.nx * args.ny, "nphase": 2, "dim": 2,
            "flux": "hll", "cfl": 0.2, "step": "one SSP-RK3 step (3 stages)",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
            "l2": flush}


# ---------------------------------------------------------------- reference arm
def oracle_step_rate(case, nsteps, warm=0):
    """The FP64 CPU oracle as it stands, on this host's cores."""
    import oracle
    g = oracle.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                    bc=case.bc)
    U = oracle.prim_to_cons(g, case.V)
    for _ in range(warm):
        U, _ = oracle.rk3_step(g, U, cfl=case.cfl)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        U, _ = oracle.rk3_step(g, U, cfl=case.cfl)
    dt = time.perf_counter() - t0
    cells = int(np.prod(case.shape))
    return cells * 3 * nsteps / dt / 1e6, dt, oracle.num_threads(), U


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
        "config": config_dict(args, 1, "n/a (CPU)"),
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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

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


def traffic_from_profile(kernel_hash):
    """DRAM bytes per sweep launch from the committed ncu summary, when it was
    taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("csrc_hash") != kernel_hash:
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

    case = make_case(args, rank)
    N, D = case.N, case.dim
    cells = int(np.prod(case.shape))
    learned = not (args.no_learned or args.profile or args.profile_pf)
    S, train_info = train_surrogate(args, dev) if learned else (None, None)

    def make_grid(precision, c=None, counters=None, scheme="c", kmodel="allaire"):
        c = c or case
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

    def timed_steps(g, K, W, c=None, dt=0.0):
        """K timed RK steps (events per step, L2 flushed in between) and the
        mean duration of the sweep launches inside them (event pairs the
        library records around each direction's launches on the same
        stream: the sweep, preceded in learned precision by the surrogate).
        dt > 0: fixed time step, else from the CFL number on the device."""
        c = c or case
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
        g, U = make_grid("fp64")
        g.set_pf_workspace(U.device)
        g.step(cfl=case.cfl, nsteps=args.warmup, tol=1e-12)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(cfl=case.cfl, nsteps=args.steps, tol=1e-12)
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

    if args.profile:
        g, U = make_grid(args.profile_precision)
        ms, sw = timed_steps(g, args.steps, args.warmup)
        print(json.dumps({"profile": True, "precision": args.profile_precision,
                          "ms_per_step": ms, "sweep_ms_per_launch": sw,
                          "steps": args.steps, "warmup": args.warmup}), flush=True)
        return 0

    # FP64 DFMA probe of this GPU (context for the derived peak below)
    peak_probe = wenoc.fp64_peak() / 1e12

    modes = ("fp64", "mixed", "learned") if learned else ("fp64", "mixed")
    results = {}
    c5 = None
    res5 = {}
    with Clocks(local) as clk:
        time.sleep(1.0)  # let the sampler start before the timed region
        for prec in modes:
            g, U = make_grid(prec)
            ms, sw = timed_steps(g, args.steps, args.warmup)
            results[prec] = (ms, sw)
            del g, U
        if learned and rank == 0:
            # the learned-weight workload: 2-D circles and shock, N = 3
            from paper_2608_00746_b300 import inputs
            c5 = inputs.circles_shock_2d(n=args.n5, seed=args.seed)
            for prec in modes:
                g, U = make_grid(prec, c5)
                res5[prec] = timed_steps(g, args.steps5, 3, c5)
                del g, U
            # the surrogate's inference kernel alone (one direction)
            g, U = make_grid("mixed", c5)
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
            infer_ms = e0.elapsed_time(e1) / 10
            infer_rows = 2 * g.ncell
            del g, U, W5
        variants = run_variants(args, rank, make_grid, timed_steps)
    clocks = clk.summary()
    # FP64 peak from unit counts and clock: 2 DFMA per clock per SM (ncu's
    # sm__sass_thread_inst_executed_op_dfma_pred_on peak_sustained = 296 per
    # cycle on 148 SMs), 2 flops each, at the maximum SM clock 2032 MHz.
    peak_fp64 = 2 * 2 * 148 * 2032e6 / 1e12

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
        return out, acc

    # matched accuracy on the headline workload
    l1s, acc2 = matched_l1(case, args.steps)
    l1 = l1s["mixed"]

    # end to end through the C ABI with host buffers: upload, step, download
    g, U = make_grid("fp64")
    host = torch.empty(U.numel(), dtype=torch.float64, pin_memory=True)
    host.copy_(U.reshape(-1).cpu())
    nbytes = U.numel() * 8
    barrier()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        g.upload(host)
        g.rk_step(cfl=case.cfl)
        g.download(host)
    e1.record(s)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / args.steps

    ms64, sw64 = results["fp64"]
    msmx, swmx = results["mixed"]
    msl = results["learned"][0] if learned else 0.0
    # max over ranks (replicas: the job takes as long as the slowest rank)
    ms64, msmx, e2e_ms, msl = replicas.max_over_ranks([ms64, msmx, e2e_ms, msl], device=dev)
    value = replicas.weak_value(ws, cells, 3, ms64)
    value_mx = replicas.weak_value(ws, cells, 3, msmx)
    e2e = replicas.weak_value(ws, cells, 3, e2e_ms)

    fl = roofline.flops_per_cell_dir(N, D, hllc=False)
    achieved = fl * cells / (sw64 * 1e-3) / 1e12
    khash = csrc_hash()
    traffic = traffic_from_profile(khash)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Mcell/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms64, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded shock-bubble initial condition)",
        "config": config_dict(args, ws, "flushed between timed steps (256 MB write)"),
        "modes": {
            "fp64": {"value": round(value, 3), "ms_per_step": round(ms64, 4)},
            "mixed": {"value": round(value_mx, 3), "ms_per_step": round(msmx, 4),
                      "speedup_vs_fp64": round(value_mx / value, 3),
                      "l1_rel_vs_fp64_max_var": l1, "l1_steps": args.steps},
        },
        "roofline": {
            "bound": "alu", "kernel": "k_sweep_win<N=2,D=2,double> (window direction sweep)",
            "achieved": round(achieved, 4), "peak": round(peak_fp64, 4), "unit": "TFLOP/s",
            "frac": round(achieved / peak_fp64, 4), "traffic": traffic,
            "peak_source": "unit count x clock: 2 DFMA/clk/SM x 2 flop x 148 SM x 2032 MHz",
            "peak_probe_measured": round(peak_probe, 4),
            "flops_per_cell_dir": fl, "sweep_ms_per_launch": round(sw64, 4),
            "sweep_ms_per_launch_mixed": round(swmx, 4),
            "hbm_bytes_per_cell_stage_min": roofline.bytes_per_cell_stage(N, D),
        },
        "clocks": clocks,
        "e2e": {"value": round(e2e, 3), "unit": "Mcell/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": args.steps * (1 + 3 * D),
        "csrc_hash": khash,
    }
    if learned:
        line["modes"]["learned"] = {
            "value": round(replicas.weak_value(ws, cells, 3, msl), 3), "ms_per_step": round(msl, 4),
            "speedup_vs_fp64": round(ms64 / msl, 3), "l1_rel_vs_fp64_max_var": l1s["learned"],
            "l1_steps": args.steps, "tau": args.tau, "accepted_face_sides": acc2,
            "ms_per_direction": round(results["learned"][1], 4)}
        line["surrogate_training"] = train_info
    if learned and rank == 0:
        l1_5, acc5 = matched_l1(c5, args.steps5)
        cells5 = int(np.prod(c5.shape))
        w5 = {}
        for prec in modes:
            ms5, sw5 = res5[prec]
            w5[prec] = {"value": round(cells5 * 3 / (ms5 * 1e-3) / 1e6, 3),
                        "ms_per_step": round(ms5, 4), "ms_per_direction": round(sw5, 4)}
            if prec != "fp64":
                w5[prec]["l1_rel_vs_fp64_max_var"] = l1_5[prec]
                w5[prec]["speedup_vs_fp64"] = round(res5["fp64"][0] / ms5, 3)
        w5["learned"]["tau"] = args.tau
        w5["learned"]["accepted_face_sides"] = acc5
        fl_row = 2 * (30 * 64 + 64 * 64 * 2 + 64 * 9)
        infer_tf = fl_row * infer_rows / (infer_ms * 1e-3) / 1e12
        w5["surrogate_inference"] = {
            "kernel": "k_mlp_fwd<SrcState<3,2>> (feature gather + 4 tcgen05 layers)",
            "rows": infer_rows, "ms_per_launch": round(infer_ms, 4),
            "achieved_tflops": round(infer_tf, 2), "flops_per_row": fl_row,
            "frac_of_bf16_measured": round(infer_tf / 1794.1, 4)}
        line["learned_workload"] = {
            "workload": f"circles_shock_2d {args.n5}x{args.n5} N=3 HLL CFL 0.2 outflow "
                        "(64 circles, radii 10-80 cells, shock ratio 1e3, seeded)",
            "steps": args.steps5, "l1_steps": args.steps5, "modes": w5}
    if variants:
        line["scheme_variants"] = variants
    if rank == 0 and not args.no_cpu_baseline:
        try:
            small = make_case(args, 0)
            v, t, cores, _ = oracle_step_rate(small, 2)
            line["cpu_baseline"] = {"value": round(v, 4), "unit": "Mcell/s", "cores": cores,
                                    "kind": "oracle", "sample": "full grid, 2 RK3 steps"}
        except Exception as e:  # the oracle must be built on the host
            line["cpu_baseline"] = {"value": None, "error": str(e)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        tdist.destroy_process_group()
    return 0


def run_variants(args, rank, make_grid, timed_steps):
    """The scheme variants, each on its own workload, FP64, same timing as the
    headline: WENO-C, WENO-CL and the WENO-W / WENO-JS comparison schemes on
    the Sec. 4.1.1 air-circle advection (n^2, dt = 0.1 n^-1, the paper's
    1e-3 at n = 100) with the consistency error after the run; the Kapila
    model on the headline shock-bubble."""
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
    g, U = make_grid("fp64", kmodel="kapila")
    ms, sw = timed_steps(g, args.steps, 3)
    cells_h = int(np.prod(g.shape))
    out["kapila"] = {"workload": "headline shock-bubble, K_p of the Kapila model",
                     "value": round(cells_h * 3 / (ms * 1e-3) / 1e6, 3),
                     "ms_per_step": round(ms, 4), "ms_per_direction": round(sw, 4)}
    del g, U
    out["phase_field"] = time_phase_field(make_grid)
    return out


def time_phase_field(make_grid, K=20):
    """Full time steps of Sec. 2.2 on the headline shock-bubble: the
    hyperbolic step, Eq. 28, the Q-map of Eq. 4 (conjugate gradients to a
    D-weighted residual of 1e-12, started from the previous step's Q) and
    the Phase-Field step, FP64; then each part timed alone."""
    import torch
    g, U = make_grid("fp64")
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
    return {"workload": "headline shock-bubble, full time step (hyperbolic + Eq. 28 + Eq. 4 + "
                        "Phase-Field step), Q-map tolerance 1e-12",
            "steps": K, "value": round(cells * 3 / (ms * 1e-3) / 1e6, 3), "unit": "Mcell/s",
            "ms_per_step": round(ms, 4), "qmap_cg_iterations_last": iters,
            "qmap_label_rounds_last": rounds, "qmap_residual_last": res,
            "qmap_unknowns_last": band, "qmap_unknowns_per_thread_last": per_thread,
            "ms_hyperbolic": round(parts[0], 4), "ms_eq28": round(parts[1], 4),
            "ms_qmap": round(parts[2], 4), "ms_pf_step": round(parts[3], 4)}


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
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
