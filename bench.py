"""Benchmark: cell-steps/s of the regularised Herschel-Bulkley time step on the
3D lid-driven cavity (256^3 cells, n=1.5, Bi=10, Re=100, Pa=1e5), every
multigrid solve to a 1e-10 relative residual.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
    python bench.py --impl reference ...   # the CPU oracle on this host's cores

Prints one JSON line (rank 0).  A step is one full pass of the method (all
stages and solves) over the whole grid.  The paper's timing protocol
(Sec. V D): a constant dt, 100 steps before the timed ones.  The cavity is
first developed from rest for --develop steps (95) by the mixed method and
checkpointed; every arm (mixed + learned, mixed alone, FP64) restarts from
that checkpoint, takes W warm-up steps and times K steps with no
instrumentation; the per-kernel event timing behind the roofline and the
stage breakdown comes from a separate instrumented pass.  Inputs live in HBM
before the timed region; every field is larger than L2, so no L2 flush is
needed between steps.
With several GPUs each rank runs an independent replica (the single-cavity
step does not shard); value = all ranks' cell-steps / the slowest rank's time.
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-steps/s at 256³ 3D HB cavity, mixed+learned vs plain FP64, same residual"
UNIT = "cell-steps/s"


# ---------------------------------------------------------------------------
# replicas: the slowest rank's time and the whole-job rate
# ---------------------------------------------------------------------------
def max_over_ranks(x, dist, device):
    """The maximum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank / seconds


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-learned", action="store_true", help="time the mixed method without the learned guess")
    ap.add_argument("--learn-n", type=int, default=128, help="cells per axis of the training cavities")
    ap.add_argument("--learn-seeds", type=int, default=6)
    ap.add_argument("--learn-steps", type=int, default=10)
    ap.add_argument("--learn-epochs", type=int, default=15)
    ap.add_argument("--vlearn-level", type=int, default=2,
                    help="multigrid level of the viscous network's training cavities (applied on the level of the "
                         "timed grid with the same cell count)")
    ap.add_argument("--vlearn-seeds", type=int, default=3)
    ap.add_argument("--vlearn-steps", type=int, default=10)
    ap.add_argument("--vlearn-epochs", type=int, default=8)
    ap.add_argument("--learn-level", type=int, default=2,
                    help="multigrid level whose nodes the network sees (0 = finest)")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip timing the plain FP64 method on the same workload")
    ap.add_argument("--workload", default="cavity256_3d_hb")
    ap.add_argument("--n", type=int, default=0, help="override cells per axis (testing only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-sweep measurement")
    ap.add_argument("--batch-only", action="store_true", help="measure only the batched sweep")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--batch-warmup", type=int, default=3)
    ap.add_argument("--batch-ncav", type=int, default=64)
    ap.add_argument("--no-batch-sequential", action="store_true",
                    help="skip timing the same cavities one context at a time")
    ap.add_argument("--develop", type=int, default=95,
                    help="steps from rest (mixed method, untimed) before the warm-up; develop + warm-up = 100 "
                         "with the default warm-up, the paper's protocol")
    ap.add_argument("--prof-steps", type=int, default=5, help="steps of the instrumented pass")
    ap.add_argument("--staged-sweep", default="0",
                    help="TMA-staged finest-level viscous sweeps: 'TX,TZ' (tile width 64 or 128, planes per block) "
                         "or 0 (hbf_set_staged_sweep)")
    ap.add_argument("--split-layout", type=int, default=1, choices=(0, 1),
                    help="colour-split layout of the FP32 finest level of the mixed viscous solve (hbf_set_split_layout)")
    ap.add_argument("--inner-drop", type=float, default=1e-3,
                    help="residual drop of each FP32 BiCGStab pass of the mixed viscous solve (hbf_set_inner_drop)")
    ap.add_argument("--staged-op", default="0",
                    help="TMA-staged finest-level viscous operator: 'ROWS,TZ' (tile 64 x ROWS, ROWS 4 or 8, planes "
                         "per block) or 0 (hbf_set_staged_op)")
    ap.add_argument("--fused-sweeps", action="store_true",
                    help="smooth the 3D FP32 finest level with the one-launch red-black sweep (hbf_set_fused_sweep)")
    ap.add_argument("--breakdown", action="store_true",
                    help="also time bottom solves, transfers, reductions, vector updates and coarse levels")
    ap.add_argument("--profiler-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(cfg_full, nsample, steps, warmup=0):
    """Time the CPU oracle on the same cavity at nsample^3 cells (a bounded
    sample of the workload: same physics and dt rule).  Returns cell-steps/s."""
    from oracle.grid import Grid
    from oracle.step import Rheology, step
    from paper_1803_00417_gb300.inputs import cavity

    name = cfg_full["name"]
    d = cfg_full["d"]
    cfg = cavity(name, n=(nsample,) * d)
    g = Grid(cfg["n"], cfg["h"], wall_u=cfg["wall_u"])
    rh = Rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    u = [np.zeros(cfg["n"]) for _ in range(d)]
    p = np.zeros(tuple(v + 1 for v in cfg["n"]))
    for _ in range(warmup):
        r = step(g, u, p, cfg["dt"], rh)
        u, p = r.u, r.p
    t0 = time.perf_counter()
    for _ in range(steps):
        r = step(g, u, p, cfg["dt"], rh)
        u, p = r.u, r.p
    dt = time.perf_counter() - t0
    return int(np.prod(cfg["n"])) * steps / dt, dt


def cpu_cores_used():
    # numpy runs the oracle's array arithmetic on one thread (no BLAS calls)
    return 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1803_00417_gb300.inputs import cavity

    cfg = cavity(args.workload)
    cfg["name"] = args.workload
    nsample = 32 if cfg["d"] == 3 else 128
    val, secs = oracle_sample(cfg, nsample, args.steps, args.warmup)
    sample = f"{nsample}^{cfg['d']} cells of the same cavity, {args.steps} timed steps after {args.warmup}"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": list(cfg["n"]), "sample_n": [nsample] * cfg["d"],
                       "precision": "fp64", "parallelism": "replicas"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cpu_cores_used(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------
SMOOTHER_DRAM_BYTES_PER_CELL = (144.20e6 + 15.16e6) / 192 ** 3  # profiles/k_visc_smooth_cavity192.md
# the colour-split form (profiles/k_visc_smooth_split_cavity192.md)
SPLIT_SMOOTHER_DRAM_BYTES_PER_CELL = (113.29e6 + 8.96e6) / 192 ** 3


def split_applies(args, prec, cfg):
    """Whether the mixed viscous solve runs its FP32 finest level in the
    colour-split layout (hbf_set_split_layout): 3D walled grid with an even x
    extent, neither the fused nor the staged sweep nor the staged operator."""
    from paper_1803_00417_gb300.hbflow import MIXED

    n = cfg["n"]
    return (prec == MIXED and args.split_layout == 1 and len(n) == 3 and n[0] % 2 == 0 and not args.fused_sweeps
            and str(args.staged_sweep) == "0" and str(args.staged_op) == "0")


def visc_smoother_bytes(d, ncell, elem, cell_eta):
    """Algorithmic bytes of one finest-level launch of the viscous smoother
    (one component, one colour): reads the other colour of u_c (ncell/2), the
    other components for the cross terms ((d-1) ncell), b_c of the colour
    (ncell/2) and the viscosity, as the cell array (ncell; the FP32 finest
    level forms the face means itself) or every face eta once (d ncell);
    writes u_c of the colour (ncell/2)."""
    return elem * ncell * (0.5 + (d - 1) + 0.5 + (1 if cell_eta else d) + 0.5)


def fused_sweep_bytes(d, ncell, elem):
    """Algorithmic bytes of one launch of the fused red-black sweep (one
    component, both colours; 3D FP32 finest level): reads u_c, the d - 1 other
    components, the cell viscosity and b_c once, writes u_c once."""
    return elem * ncell * (1 + (d - 1) + 1 + 1 + 1)


def run_batch_sweep(args, clocks=None):
    """64 seeded 2D cavities (sizes 128..512, random Bi, n, Re) advanced together
    by the batched step in mixed precision, after the tiling autotuner; then the
    same cavities advanced one context at a time for comparison."""
    import torch

    from paper_1803_00417_gb300.hbflow import MIXED, Batch, HBFlow
    from paper_1803_00417_gb300.inputs import batch_sweep

    cfgs = batch_sweep(ncav=args.batch_ncav, seed=0)
    cells = int(sum(np.prod(c["n"]) for c in cfgs))
    B = Batch([c["n"] for c in cfgs], [c["h"] for c in cfgs], [c["wall_u"] for c in cfgs], precision=MIXED)
    for i, c in enumerate(cfgs):
        v = B.cavity(i)
        v.set_rheology(c["K"], c["nexp"], c["tau_y"], c["m"])
        v.set_solver(rtol=1e-10, max_cycles=200)
        v.set_field("U", np.zeros(2 * int(np.prod(c["n"]))))
        v.set_field("P", np.zeros(int(np.prod([s + 1 for s in c["n"]]))))
    B.set_dt([c["dt"] for c in cfgs])
    t0 = time.perf_counter()
    tuned = B.autotune(reps=3)
    tune_s = time.perf_counter() - t0
    for _ in range(args.batch_warmup):
        B.step()
    B.sync()
    n0 = B.launch_count()
    cyc = {"mac": 0, "visc": 0, "nodal": 0}
    conv = 0
    if clocks is not None:
        clocks.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.batch_steps):
        st = B.step()
        for s in st:
            for k in cyc:
                cyc[k] += s[k]["cycles"]
            conv += int(all(s[k]["converged"] for k in cyc))
    B.sync()
    secs = time.perf_counter() - t0
    clk = clocks.stop() if clocks is not None else None
    launches = B.launch_count() - n0
    tiling = B.tiling()
    B.profile(True)
    for _ in range(2):
        B.step()
    phases = B.profile_read()
    B.profile(False)
    out = {"value": cells * args.batch_steps / secs, "unit": UNIT, "ms_per_step": 1e3 * secs / args.batch_steps,
           "steps": args.batch_steps, "warmup": args.batch_warmup, "precision": "mixed", "rtol": 1e-10,
           "workload": f"{len(cfgs)} 2D lid-driven cavities, sizes {{128,256,384,512}}^2 (seed 0), Bi U[0,50], "
                       f"n U[0.3,1.5], Re log-U[1,1000], m=1e4, dt=0.5h each, from rest",
           "cells": cells, "tiling": tiling, "autotune": dict(tuned, seconds=tune_s),
           "launches_per_step": launches / args.batch_steps,
           "converged_solves": f"{conv}/{len(cfgs) * args.batch_steps}",
           "cycles_per_cavity_step": {k: v / (len(cfgs) * args.batch_steps) for k, v in cyc.items()},
           "timer": "host wall clock around the steps (each step synchronises on its residual norms)",
           "phases_2_steps": phases,
           "clocks": clk}
    B.close()
    if not args.no_batch_sequential:
        sims = []
        for c in cfgs:
            s_ = HBFlow(c["n"], c["h"], c["wall_u"], precision=MIXED)
            s_.set_rheology(c["K"], c["nexp"], c["tau_y"], c["m"])
            s_.set_solver(rtol=1e-10, max_cycles=200)
            s_.set_field("U", np.zeros(2 * int(np.prod(c["n"]))))
            s_.set_field("P", np.zeros(int(np.prod([v + 1 for v in c["n"]]))))
            sims.append(s_)
        for _ in range(args.batch_warmup):
            for s_, c in zip(sims, cfgs):
                s_.step(c["dt"])
        torch.cuda.synchronize()
        n0 = sum(s_.launch_count() for s_ in sims)
        t0 = time.perf_counter()
        for _ in range(args.batch_steps):
            for s_, c in zip(sims, cfgs):
                s_.step(c["dt"])
        torch.cuda.synchronize()
        secs1 = time.perf_counter() - t0
        nl = sum(s_.launch_count() for s_ in sims) - n0
        for s_ in sims:
            s_.close()
        seq = cells * args.batch_steps / secs1
        out["sequential_contexts"] = {"value": seq, "unit": UNIT, "ms_per_step": 1e3 * secs1 / args.batch_steps,
                                      "launches_per_step": nl / args.batch_steps}
        out["speedup_vs_sequential"] = out["value"] / seq
    return out


def run_ours(args):
    import torch

    from paper_1803_00417_gb300 import build
    from paper_1803_00417_gb300.hbflow import FP64, MIXED, HBFlow
    from paper_1803_00417_gb300.inputs import cavity

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        build.build()
    if dist is not None:
        dist.barrier()

    if args.batch_only:
        if rank == 0:
            res = run_batch_sweep(args, Clocks(local))
            print(json.dumps({"batch_sweep": res}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    over = {"n": (args.n,) * 3} if args.n else {}
    cfg = cavity(args.workload, **over)
    cfg["name"] = args.workload
    d = cfg["d"]
    ncell = int(np.prod(cfg["n"]))
    prec = MIXED if args.precision == "mixed" else FP64
    learned = None
    model = None
    vmodel = None
    vlev = None
    if prec == MIXED and not args.no_learned:
        # offline part of the learned guess: solver-generated pairs on small
        # cavities of the same family, trained by the library's kernels
        from paper_1803_00417_gb300.hbflow import UNet
        from paper_1803_00417_gb300.learned import box_mask, coarse_cells, generate_pairs, net_box, train

        t0 = time.perf_counter()
        lv = args.learn_level
        ln = (args.learn_n,) * d
        xs, ys, _ = generate_pairs(ln, seeds=range(args.learn_seeds), steps=args.learn_steps, precision=MIXED,
                                   level=lv)
        lbox = net_box(coarse_cells(ln, lv))
        tnet = UNet(lbox, train=True, seed=0)
        hist = train(tnet, xs, ys, box_mask(coarse_cells(ln, lv), lbox), epochs=args.learn_epochs, lr=1e-3,
                     batch=4)
        params = tnet.get_params()
        tnet.close()
        model = UNet(net_box(coarse_cells(cfg["n"], lv)), train=False)
        model.set_params(params)
        learned = {"nodal": {"train_cavities": f"{args.learn_seeds} x {args.learn_n}^{d}, random Bi/n/Re",
                             "train_pairs": int(len(xs)), "level": lv,
                             "epochs": args.learn_epochs, "loss_first": hist[0], "loss_last": hist[-1],
                             "box": list(net_box(coarse_cells(cfg["n"], lv)))}}
        # the viscous network: pairs from cavities with the previous-increment
        # step on, restricted to a level whose cell count the timed grid has
        # one level further down (128^3 level 2 = 256^3 level 3 = 32^3 cells)
        from paper_1803_00417_gb300.learned import cell_box, cell_mask, generate_visc_pairs

        vl = args.vlearn_level
        nvl = coarse_cells(ln, vl)
        vlev = next((l for l in range(12) if coarse_cells(cfg["n"], l) == nvl), None)
        if vlev is not None:
            vxs, vys, _ = generate_visc_pairs(ln, seeds=range(args.vlearn_seeds), steps=args.vlearn_steps,
                                              level=vl)
            vbox = cell_box(nvl)
            vnet = UNet(vbox, train=True, seed=1)
            vhist = train(vnet, vxs, vys, cell_mask(nvl, vbox), epochs=args.vlearn_epochs, lr=1e-3, batch=4)
            vmodel = UNet(vbox, train=False)
            vmodel.set_params(vnet.get_params())
            vnet.close()
            learned["viscous"] = {"train_cavities": f"{args.vlearn_seeds} x {args.learn_n}^{d}, random Bi/n/Re",
                                  "train_pairs": int(len(vxs)), "train_level": vl, "level": vlev,
                                  "epochs": args.vlearn_epochs, "loss_first": vhist[0], "loss_last": vhist[-1],
                                  "box": list(vbox)}
        learned["offline_seconds"] = time.perf_counter() - t0
    sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=prec)
    sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    sim.set_solver(rtol=1e-10, max_cycles=200)
    sim.set_fused_sweep(args.fused_sweeps)
    staged = [int(v) for v in str(args.staged_sweep).split(",")] if args.staged_sweep != "0" else [0, 16]
    sim.set_staged_sweep(staged[0], staged[1] if len(staged) > 1 else 16)
    sop = [int(v) for v in str(args.staged_op).split(",")] if args.staged_op != "0" else [0, 16]
    sim.set_staged_op(sop[0], sop[1] if len(sop) > 1 else 16)
    if prec == MIXED:
        sim.set_inner_drop(args.inner_drop)
        sim.set_split_layout(args.split_layout)
    zeros_u = np.zeros(d * ncell)
    zeros_p = np.zeros(int(np.prod([v + 1 for v in cfg["n"]])))
    sim.set_field("U", zeros_u)
    sim.set_field("P", zeros_p)
    dt = cfg["dt"]
    stream = torch.cuda.current_stream()
    # develop the flow from rest (untimed, no learned guess), checkpoint it
    t0 = time.perf_counter()
    for _ in range(args.develop):
        sim.step(dt)
    developed = sim.get_state()
    develop_s = time.perf_counter() - t0
    if model is not None:
        from paper_1803_00417_gb300.hbflow import set_guess_model, set_visc_guess_model

        set_guess_model(sim, model, args.learn_level)
        sim.set_visc_guess(2 if vmodel is not None else 1)
        if vmodel is not None:
            set_visc_guess_model(sim, vmodel, vlev)

    def restart(sim_):
        rec, u_, p_ = developed
        sim_.set_state(rec, u_, p_)

    def timed(sim_, level, clocks_=None, profiler_range=False):
        restart(sim_)
        for _ in range(args.warmup):
            sim_.step(dt)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        sim_.profile_enable(level)
        n0 = sim_.launch_count()
        cyc = {"mac": 0, "visc": 0, "nodal": 0}
        conv = True
        used = 0
        vused = [0, 0]
        torch.cuda.synchronize()
        if clocks_ is not None:
            clocks_.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if profiler_range:
            torch.cuda.profiler.start()
        e0.record(stream)
        for _ in range(args.steps):
            st = sim_.step(dt)
            for k in cyc:
                cyc[k] += st[k]["cycles"]
                conv &= st[k]["converged"]
            used += int(st["nodal"]["guess"])
            vused[0] += st["visc"]["guess"] & 1
            vused[1] += (st["visc"]["guess"] >> 1) & 1
        e1.record(stream)
        torch.cuda.synchronize()
        if profiler_range:
            torch.cuda.profiler.stop()
        clk_ = clocks_.stop() if clocks_ is not None else None
        ms_ = e0.elapsed_time(e1)
        nl = sim_.launch_count() - n0
        prof_ = {k: sim_.profile_read(k) for k in sim_.PROFILE_SLOTS}
        sim_.profile_enable(0)
        ms_ = max_over_ranks(ms_, dist, "cuda")
        timed.guess_used = used
        timed.vguess_used = vused
        return ms_, cyc, conv, nl, prof_, clk_

    clocks = Clocks(local)
    ms, cycles, converged, launches, _, clk = timed(sim, 0, clocks, args.profiler_range)
    value = job_rate(world, ncell * args.steps, ms / 1e3)
    if learned is not None:
        learned["nodal"]["guess_accepted_steps"] = f"{timed.guess_used}/{args.steps}"
        learned["viscous_steps_taken"] = {"previous_increment": f"{timed.vguess_used[0]}/{args.steps}",
                                          "network": f"{timed.vguess_used[1]}/{args.steps}"}
    # instrumented pass: CUDA events around every finest-level launch of the
    # main kernel classes (level 2: every class) for the roofline and the
    # stage breakdown, continuing from the timed steps' state
    lvl = 2 if args.breakdown else 1
    sim.profile_enable(lvl)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.prof_steps):
        sim.step(dt)
    e1.record(stream)
    torch.cuda.synchronize()
    prof_ms = e0.elapsed_time(e1) / args.prof_steps
    prof = {k: sim.profile_read(k) for k in sim.PROFILE_SLOTS}
    sim.profile_enable(0)

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not args.no_e2e:
        hu = torch.empty(d * ncell, dtype=torch.float64, pin_memory=True).numpy()
        hp = torch.empty(zeros_p.size, dtype=torch.float64, pin_memory=True).numpy()
        sim.get_field("U", hu)
        sim.get_field("P", hp)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sim.set_field("U", hu)
            sim.set_field("P", hp)
            sim.step(dt)
            sim.get_field("U", hu)
            sim.get_field("P", hp)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        secs = max_over_ranks(secs, dist, "cuda")
        e2e = {"value": job_rate(world, ncell * args.e2e_steps, secs), "unit": UNIT,
               "h2d_bytes_per_step": int(hu.nbytes + hp.nbytes), "d2h_bytes_per_step": int(hu.nbytes + hp.nbytes)}

    mixed_only = None
    increment_only = None
    if model is not None:
        # the same method without the networks: the previous-increment step of
        # the viscous guess alone, then no guess at all (the V-cycles and
        # iterations saved, and what each part costs)
        set_guess_model(sim, None)
        set_visc_guess_model(sim, None)
        sim.set_visc_guess(1)
        msi, cyci, convi, _, _, _ = timed(sim, 0)
        increment_only = {"value": world * ncell * args.steps / (msi / 1e3), "unit": UNIT,
                          "ms_per_step": msi / args.steps, "converged": bool(convi),
                          "cycles_per_step": {k: v / args.steps for k, v in cyci.items()},
                          "guess": "viscous solve: previous-increment step only; no network"}
        sim.set_visc_guess(0)
        msm, cycm, convm, _, _, _ = timed(sim, 0)
        mixed_only = {"value": world * ncell * args.steps / (msm / 1e3), "unit": UNIT,
                      "ms_per_step": msm / args.steps, "converged": bool(convm),
                      "cycles_per_step": {k: v / args.steps for k, v in cycm.items()},
                      "guess": "none (the solves start from u^m and p^{m-1/2})"}
        model.close()
        if vmodel is not None:
            vmodel.close()

    fp64 = None
    if prec == MIXED and not args.no_fp64_compare:
        sim.close()
        ref = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=FP64)
        ref.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
        ref.set_solver(rtol=1e-10, max_cycles=200)
        ms64, cyc64, conv64, _, _, _ = timed(ref, 0)
        ref.close()
        v64 = world * ncell * args.steps / (ms64 / 1e3)
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / args.steps,
                "cycles_per_step": {k: v / args.steps for k, v in cyc64.items()}, "converged": bool(conv64),
                "speedup_of_value": value / v64,
                "note": "plain FP64 method (FP64 V-cycles, FP64 BiCGStab), same workload, residual, protocol "
                        "and developed state, no instrumentation"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    elem = 4 if prec == MIXED else 8
    sm_ms, sm_n = prof["visc_smooth"]
    # the guess slot times whole sections whose launches also count in their
    # own slots: reported beside the stages, not in their sum
    guess_ms = prof["guess"][0] / args.prof_steps if prof["guess"][1] > 0 else None
    stages = {k: v[0] / args.prof_steps for k, v in prof.items() if v[1] > 0 and k != "guess"}
    roofline = None
    if sm_n > 0:
        per_launch_s = sm_ms / sm_n / 1e3
        fused = prec == MIXED and d == 3 and args.fused_sweeps
        split = split_applies(args, prec, cfg)
        algo = fused_sweep_bytes(d, ncell, elem) if fused else visc_smoother_bytes(d, ncell, elem, prec == MIXED)
        ach = algo / per_launch_s / 1e9
        # DRAM bytes per cell of this kernel from one full ncu capture at 192^3
        # of the current kernel (profiles/k_visc_smooth_cavity192.md), scaled
        # to this grid by the cell count (the kernel reads the same arrays per
        # cell at any size; the 256^3 workload is too large to capture)
        per_cell = SPLIT_SMOOTHER_DRAM_BYTES_PER_CELL if split else SMOOTHER_DRAM_BYTES_PER_CELL
        traffic = per_cell * ncell if (prec == MIXED and not fused and per_cell) else None
        roofline = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                    "traffic": traffic,
                    "traffic_source": f"ncu capture of the same kernel at 192^3 ({per_cell:.1f} B/cell), scaled by cells"
                    if traffic else None,
                    "kernel": "k_visc_sweep_rb (fused red-black sweep, finest level)" if fused
                    else ("k_visc_smooth_split (finest level, colour-split layout)" if split
                          else "k_visc_smooth (finest level)"),
                    "launches": sm_n, "avg_launch_us": per_launch_s * 1e6,
                    "algorithmic_bytes_per_launch": algo,
                    "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}

    cpu = None
    if not args.no_cpu:
        # about 10 s of oracle work on the host (a 32^3 step takes about 1 s)
        nsample, nsteps = (32, 10) if d == 3 else (128, 10)
        val, secs = oracle_sample(cfg, nsample, nsteps)
        cpu = {"value": val, "unit": UNIT, "cores": cpu_cores_used(), "kind": "oracle",
               "sample": f"{nsteps} steps from rest of the same cavity at {nsample}^{d} cells ({secs:.1f} s)"}

    batch = None
    if not args.no_batch:
        batch = run_batch_sweep(args, clocks)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == FP64 else ("f64+f32+bf16" if learned else "f64+f32"), "data": "synthetic",
            "config": {"workload": args.workload, "n": list(cfg["n"]),
                       "precision": args.precision + ("+learned" if learned else ""),
                       "rtol": 1e-10, "dt": dt, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "no flush: every field (>= 134 MB) exceeds the 129 MB L2",
                       "viscous_sweeps": ("one-launch fused" if args.fused_sweeps else
                                          f"TMA-staged {staged[0]}x8 tiles, {staged[1]} planes per block"
                                          if staged[0] else "two launches per component, unstaged"),
                       "inner_drop": args.inner_drop if prec == MIXED else None,
                       "finest_fp32_layout": ("colour-split" if split_applies(args, prec, cfg) else "natural")
                       if prec == MIXED else None,
                       "viscous_operator": (f"TMA-staged 64x{sop[0]} tiles, {sop[1]} planes per block" if sop[0]
                                            else "unstaged, one thread per cell"),
                       "cycles_per_step": {k: v / args.steps for k, v in cycles.items()},
                       "converged": bool(converged)},
            "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "fp64_method": fp64, "learned_guess": learned, "mixed_without_learned": mixed_only,
            "mixed_previous_increment_only": increment_only,
            "batch_sweep": batch,
            "clocks": clk,
            "protocol": {"develop_steps": args.develop, "develop_seconds": develop_s, "warmup": args.warmup,
                         "timed_steps": args.steps, "instrumentation": "none in the timed steps"},
            "stage_ms_per_step": stages,
            "learned_guess_ms_per_step": guess_ms,
            "instrumented_pass": {"steps": args.prof_steps, "level": lvl, "ms_per_step": prof_ms,
                                  "stages_sum_ms": sum(stages.values()),
                                  "stages_share": sum(stages.values()) / prof_ms}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
