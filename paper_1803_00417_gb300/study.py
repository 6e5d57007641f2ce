"""Experiments of the paper re-run on the library (marshalling and control
only: every step and every diagnostic runs in the CUDA library).

    python -m paper_1803_00417_gb300.study cessation   [--n 256] [--dt 1e-5]
    python -m paper_1803_00417_gb300.study sweep       [--n 128] [--dt 4e-5]
    python -m paper_1803_00417_gb300.study cessation3d [--n 64]  [--dt 4e-5]
    python -m paper_1803_00417_gb300.study rate        [--sizes 32,64,128,256]

* ``cessation`` (Sec. IV): the 2D lid-driven cavity, Bingham, Re = 1, Bi = 10,
  Pa = 400, started from rest.  The steady criterion (Sec. III A, 1e-5) is
  evaluated after every step; at the time the paper stops the lid
  (t = 0.0205552) the state is checkpointed, the lid is stopped and the run
  continues until no cell is yielded: t_c, beside the paper's 1.2844e-3.
  Each cessation runs with the Crank-Nicolson weighting throughout and with
  the first steps after the stop taken by backward Euler (``--damp``).
  Yield zones (stagnant / plug) are reported at the paper's snapshot times
  of the start-up and of the cessation.
* ``sweep`` (Sec. IV, V A): steady states of 2D cavities (Bingham at several
  Bi, Herschel-Bulkley with n = 0.5 and 1.5), each with its primary vortex
  centre, the extremum of the stream function, and centre-line profiles
  u_x(x = 1/2, y) and u_y(x, y = 1/2).
* ``cessation3d`` (Sec. V C): the same start-up / cessation study in the 3D
  cavity (lid +x on the top wall), yield zones and t_c.
* ``rate`` (Sec. V D): cell-steps per second of the 3D Bingham cavity
  (Re = 1, Bi = 10) against the cells per axis, with the paper's timing
  protocol: constant dt, 100 warm-up steps, the mean of the next 10.

Every result is one JSON line on stdout (and appended to ``--out`` if given).
"""

import argparse
import json
import sys
import time

import numpy as np

from .hbflow import FP64, MIXED, HBFlow
from .inputs import cavity

T_STOP = 0.0205552     # Sec. IV: the lid is stopped at this time
T_C_PAPER = 1.2844e-3  # Sec. IV: the paper's cessation time for this case
STARTUP_SNAPSHOTS = (3.5e-6, 1.05e-5, 9.33e-5, 9.54e-4)
CESSATION_SNAPSHOTS = (3.89e-5, 6.48e-4, 1.1664e-3, 1.2729e-3)


def emit(rec, out=None):
    line = json.dumps(rec)
    print(line, flush=True)
    if out:
        with open(out, "a") as f:
            f.write(line + "\n")


def make(n, precision=FP64, **over):
    cfg = cavity(tuple(n), **over)
    sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=precision)
    sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    d = len(cfg["n"])
    sim.set_velocity([np.zeros(cfg["n"]) for _ in range(d)])
    sim.set_pressure(np.zeros(tuple(v + 1 for v in cfg["n"])))
    return sim, cfg


def zone_summary(sim):
    y = sim.yield_info()
    ncell = sim.ncell
    return dict(yielded_frac=y["yielded"] / ncell, tau_max=y["tau_max"],
                stagnant_frac=y["cells"]["stagnant"] / ncell, plug_frac=y["cells"]["plug"] / ncell,
                zones=y["zones"])


def steps_for(t, dt):
    return int(round(t / dt))


def startup(sim, dt, t_stop, snapshots, tol=1e-5):
    """Step from rest to t_stop; the first time the steady criterion holds,
    and the zones at the snapshot times (nearest step)."""
    nsteps = steps_for(t_stop, dt)
    marks = {max(1, steps_for(t, dt)): t for t in snapshots}
    t_steady, snaps, last_change = None, [], None
    t0 = time.time()
    for m in range(1, nsteps + 1):
        sim.step(dt)
        last_change = sim.step_change()
        if t_steady is None and last_change < tol:
            t_steady = m * dt
        if m in marks:
            snaps.append(dict(t_paper=marks[m], t=m * dt, **zone_summary(sim)))
    return dict(steps=nsteps, t=nsteps * dt, t_steady_criterion=t_steady, last_change=last_change,
                wall_s=time.time() - t0, snapshots=snaps)


FRACTIONS = (1e-2, 1e-3, 1e-4)


def cessation_from(sim, dt, snapshots, max_steps, damp_steps=0):
    """t_c from the current state (native driver); then, from the same state
    restored from a checkpoint, the zones at the snapshot times and the first
    times at which the yielded cells fall below the FRACTIONS of the box
    (the strict criterion, no yielded cell at all, turns on the last few
    cells, whose |tau| can hover within 0.1% of tau_y for many steps).  The
    state is restored again at the end.  damp_steps: backward-Euler steps
    right after the lid stops (see hbf_run_cessation)."""
    rec, u, p = sim.get_state()
    t0 = time.time()
    r = sim.run_cessation(dt, max_steps=max_steps, damp_steps=damp_steps)
    wall = time.time() - t0
    sim.set_state(rec, u, p)
    d = sim.d
    sim.set_walls(np.zeros((d, 2, d)))
    marks = {steps_for(t, dt): t for t in snapshots}
    last = max(max(marks), r["steps"] if r["reached"] else max_steps)
    snaps, t_frac, hist = [], {}, []
    for m in range(1, last + 1):
        sim.set_theta(1.0 if m <= damp_steps else 0.5)
        sim.step(dt)
        sim.set_theta(0.5)
        z = zone_summary(sim)
        hist.append((z["yielded_frac"], z["tau_max"]))
        for f in FRACTIONS:
            if f not in t_frac and z["yielded_frac"] < f:
                t_frac[f] = m * dt
        if m in marks:
            snaps.append(dict(t_paper=marks[m], t=m * dt, **z))
    sim.set_state(rec, u, p)
    every = max(1, len(hist) // 200)
    return dict(damp_steps=damp_steps, steps=r["steps"], t_c=r["t_c"], t_c_interp=r["t_c_interp"],
                reached=bool(r["reached"]), tau_ratio=r["tau_ratio"], wall_s=wall, snapshots=snaps,
                t_yielded_below={str(f): t_frac.get(f) for f in FRACTIONS},
                history=dict(every_steps=every, yielded_frac=[h[0] for h in hist[::every]],
                             tau_max=[h[1] for h in hist[::every]]))


def run_cessation_study(args):
    for dt in args.dt:
        sim, cfg = make((args.n, args.n), FP64, Re=1.0, Bi=10.0, Pa=400.0, nexp=1.0)
        st = startup(sim, dt, T_STOP, STARTUP_SNAPSHOTS)
        at_stop = zone_summary(sim)
        vort = sim.vortex()
        ces = [cessation_from(sim, dt, CESSATION_SNAPSHOTS, steps_for(20 * T_C_PAPER, dt), k) for k in args.damp]
        for ce in ces:
            ce["t_c_rel_diff"] = (ce["t_c_interp"] - T_C_PAPER) / T_C_PAPER if ce["reached"] else None
            ce["t_1e-3_rel_diff"] = ((ce["t_yielded_below"]["0.001"] - T_C_PAPER) / T_C_PAPER
                                     if ce["t_yielded_below"]["0.001"] else None)
        emit(dict(study="cessation", workload=f"cavity{args.n}_bingham_Re1_Bi10_Pa400", dt=dt,
                  startup=st, at_lid_stop=dict(vortex=vort, **at_stop), cessation=ces,
                  t_c_paper=T_C_PAPER), args.out)
        sim.close()


SWEEP = [
    dict(name="bingham_Re1_Bi1", Re=1.0, Bi=1.0, nexp=1.0),
    dict(name="bingham_Re1_Bi10", Re=1.0, Bi=10.0, nexp=1.0),
    dict(name="hb_n0.5_Re1_HB1", Re=1.0, Bi=1.0, nexp=0.5),
    dict(name="hb_n1.5_Re1_HB1", Re=1.0, Bi=1.0, nexp=1.5),
]


def run_sweep(args):
    for case in SWEEP:
        sim, cfg = make((args.n, args.n), FP64, Re=case["Re"], Bi=case["Bi"], Pa=400.0, nexp=case["nexp"])
        t0 = time.time()
        r = sim.run_steady(args.dt, tol=1e-5, max_steps=args.max_steps)
        v = sim.vortex()
        prof_u = sim.centreline(0, 1).tolist()   # u_x along y at x = 1/2
        prof_v = sim.centreline(1, 0).tolist()   # u_y along x at y = 1/2
        emit(dict(study="sweep", case=case["name"], n=args.n, dt=args.dt, steady=r,
                  vortex_centre=v["centre"], psi_extremum=v["psi"], zones=zone_summary(sim),
                  wall_s=time.time() - t0,
                  profiles=dict(u_x_vertical_centreline=prof_u, u_y_horizontal_centreline=prof_v)), args.out)
        sim.close()


def run_cessation3d(args):
    dt = args.dt[0]
    sim, cfg = make((args.n,) * 3, MIXED if args.mixed else FP64, Re=1.0, Bi=10.0, Pa=400.0, nexp=1.0)
    st = startup(sim, dt, T_STOP, STARTUP_SNAPSHOTS)
    at_stop = zone_summary(sim)
    vort = sim.vortex()
    ce = [cessation_from(sim, dt, CESSATION_SNAPSHOTS, steps_for(20 * T_C_PAPER, dt), k) for k in args.damp]
    emit(dict(study="cessation3d", workload=f"cavity{args.n}^3_bingham_Re1_Bi10_Pa400", dt=dt,
              precision="mixed" if args.mixed else "fp64", startup=st,
              at_lid_stop=dict(vortex_centre_plane_y_half=vort, **at_stop), cessation=ce), args.out)
    sim.close()


def run_rate(args):
    import torch

    for n in args.sizes:
        for prec, pname in ((FP64, "fp64"), (MIXED, "mixed")):
            sim, cfg = make((n,) * 3, prec, Re=1.0, Bi=10.0, Pa=400.0, nexp=1.0)
            dt = cfg["dt"]  # constant: CFL 0.5 against the unit lid speed
            for _ in range(args.warmup):
                sim.step(dt)
            stream = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                sim.step(dt)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            emit(dict(study="rate", n=n, cells=n ** 3, precision=pname, warmup=args.warmup, steps=args.steps,
                      ms_per_step=ms, cell_steps_per_s=n ** 3 / (ms * 1e-3)), args.out)
            sim.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("study", choices=["cessation", "sweep", "cessation3d", "rate"])
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--dt", type=str, default="")
    ap.add_argument("--max-steps", type=int, default=20000)
    ap.add_argument("--sizes", type=str, default="32,64,128,256")
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--mixed", action="store_true")
    ap.add_argument("--damp", type=str, default="0,2,100000",
                    help="cessation variants: backward-Euler steps right after the lid stops")
    ap.add_argument("--out", type=str, default="")
    args = ap.parse_args(argv)
    from . import build

    build.build()
    defaults = dict(cessation=(256, "1e-5"), sweep=(128, "4e-5"), cessation3d=(64, "4e-5"), rate=(0, "0"))
    n0, dt0 = defaults[args.study]
    args.n = args.n or n0
    args.dt = [float(v) for v in (args.dt or dt0).split(",")]
    if args.study == "sweep":
        args.dt = args.dt[0]
    args.sizes = [int(v) for v in args.sizes.split(",")]
    args.damp = [int(v) for v in args.damp.split(",")]
    dict(cessation=run_cessation_study, sweep=run_sweep, cessation3d=run_cessation3d, rate=run_rate)[args.study](args)
    return 0


if __name__ == "__main__":
    sys.exit(main())
