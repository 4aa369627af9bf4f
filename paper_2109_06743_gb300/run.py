"""Production run of a named workload on one GPU: ``python -m
paper_2109_06743_gb300.run --workload asym_1024x512_v12 --steps 2000``.

Every ``--every`` steps it prints one JSON line with the time, the energy
partition (kinetic+thermal of each species, electric, magnetic; Sec. 3.2's
energy accounting), the total-energy drift, each species' mass and the
reconnected flux on the X line (GEM diagnostic, Sec. 3.3) with the
reconnection rate since the previous line, the step time and the Newton
iterations per fit; the steps are FP32 f with the moment fit (Algorithm 1),
warm-started by a network trained on a smaller run of the same velocity grid
unless ``--no-mlp``, and with ``--retrain-every K`` retrained on the run's
own fits every K steps. ``--save PATH`` writes a checkpoint at the end (and
every ``--save-every`` steps); ``--resume PATH`` continues a run from one
(its network travels in the checkpoint, so no new training; the energy
drift is then counted from the resumed state)."""
import argparse
import json
import sys
import time

import numpy as np
import torch

from . import abi, build
from . import workloads as W
from .driver import Simulation


def diagnostics(sim, cfg, yl):
    kin, ee, eb = sim.energies()
    mass = [float(m[:, 0].sum().item()) for m in sim.mom_t]
    return [float(x) for x in kin] + [float(ee), float(eb)], mass, sim.reconnected_flux(yl)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="asym_1024x512_v12", choices=sorted(W.NAMED))
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--no-mlp", action="store_true")
    ap.add_argument("--retrain-every", type=int, default=0,
                    help="retrain the warm-start network on the run's own fits every this many steps (0: never)")
    ap.add_argument("--out", default=None, help="also write the lines to this file")
    ap.add_argument("--save", default=None, help="checkpoint file written at the end (Simulation.save)")
    ap.add_argument("--save-every", type=int, default=0, help="also write the checkpoint every this many steps")
    ap.add_argument("--resume", default=None, help="continue from this checkpoint instead of the initial state")
    args = ap.parse_args(argv)
    build.build()
    abi.lib()
    device = "cuda:0"
    mlp = None
    if args.resume:
        sim = Simulation.resume(args.resume, device=device)
        cfg = sim.cfg
        if not args.no_mlp:
            try:
                mlp = abi.mlp_get_weights(sim.ctx)
            except abi.VlasovError:
                mlp = None  # the checkpoint has no network: cold-started fits
    else:
        if not args.no_mlp:
            from .warmstart import train_warm_start
            mlp, info = train_warm_start(W.TRAIN_FROM[args.workload], device)
        cfg = W.named(args.workload, precision=32)
        sim = Simulation(cfg, W.initial_state(cfg, np.float32), None, W.initial_yee(cfg), device=device)
        if mlp is not None:
            abi.mlp_set_weights(sim.ctx, mlp)
    yl = W.x_line(cfg)
    e0, m0, psi_prev = diagnostics(sim, cfg, yl)
    E0 = sum(e0)
    out = open(args.out, "w") if args.out else None
    t_prev, wall = sim.time, time.perf_counter()
    first = {"workload": cfg.name if args.resume else args.workload, "step": sim.nstep, "x_line_y": yl, "dt": cfg.dt,
             "channels": ["kinetic+thermal " + s.name for s in cfg.species] + ["electric", "magnetic"],
             "energy": e0, "mass": m0, "reconnected_flux": psi_prev, "mlp": mlp is not None}
    for line in (first,):
        print(json.dumps(line), flush=True)
        if out:
            out.write(json.dumps(line) + "\n")
    nfit = 2 * cfg.ncell * len(cfg.species)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev0.record(sim.stream)
    st_prev, k_prev = np.array(sim.stats(), dtype=np.float64), sim.nstep
    retrains = []
    k0 = sim.nstep
    for k in range(k0 + 1, k0 + args.steps + 1):
        if mlp is not None and args.retrain_every > 0 and k % args.retrain_every == 0:
            from .warmstart import retrain
            retrains.append(retrain(sim))  # this step runs with the harvest on
        else:
            sim.step(use_mlp=mlp is not None)
        if args.save and args.save_every > 0 and k % args.save_every == 0:
            sim.save(args.save)
        if k % args.every == 0 or k == k0 + args.steps:
            ev1 = torch.cuda.Event(enable_timing=True)
            ev1.record(sim.stream)
            e, m, psi = diagnostics(sim, cfg, yl)
            t = sim.time
            st = np.array(sim.stats(), dtype=np.float64)
            d, nk = st - st_prev, k - k_prev
            line = {"step": k, "t": t, "energy": e, "energy_fraction": [x / sum(e) for x in e],
                    "energy_drift": sum(e) / E0 - 1.0, "mass_rel_change": [a / b - 1.0 for a, b in zip(m, m0)],
                    "reconnected_flux": psi, "reconnection_rate": (psi - psi_prev) / (t - t_prev),
                    "ms_per_step": ev0.elapsed_time(ev1) / nk,
                    "newton_iterations_per_fit": d[0] / (nfit * nk), "slow_evaluations_per_fit": d[6] / (nfit * nk),
                    "newton_fallbacks": int(st[1]), "clipped_cells_in_interval": int(d[2]), "retrains": len(retrains),
                    "wall_s": time.perf_counter() - wall}
            psi_prev, t_prev, st_prev, k_prev = psi, t, st, k
            ev0 = torch.cuda.Event(enable_timing=True)
            ev0.record(sim.stream)
            print(json.dumps(line), flush=True)
            if out:
                out.write(json.dumps(line) + "\n")
    torch.cuda.synchronize()
    if args.save:
        sim.save(args.save)
    sim.close()
    if out:
        out.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
