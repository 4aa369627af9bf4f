"""Benchmark of the moment-fitting PFC Vlasov hot path (arXiv:2109.06743).

One step = one full time step of Algorithm 1 (Sec. 2.2) over the whole
workload: field half step, fused x+y PFC sweep, velocity PFC pass with fused
moments, SSP-RK3 ten-moment fluid step, Newton fits of the V and F
Maxwellians, exchange + limiter with fused moments, field half step, for
both species. Inputs are synthetic (seeded Harris sheet, paper Sec. 3.3
structure) and resident in HBM when the timed region starts; f (4.3 GB at
the default size) is far larger than the 129 MB L2, so no flush is needed.

The headline form is the paper's solver in FP32 with the Newton fits
started from the warm-start network (FP32+MLP): the network is trained on
the GPU during set-up, outside the timed region, on the converged fits of a
cold-started 128 x 64 run with the same velocity grid; the line also reports
the same steps with cold-started fits and the plain FP64 form.

Metric: phase-space cell updates per second = (sum over species of
spatial cells x velocity cells) x steps / time, over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (oracle/, the baseline of this
project; the paper has no code) on a bounded sample of the same workload on
the host cores. Under torchrun each rank runs an independent replica
(replicas only: the method's spatial decomposition is not needed on one
GPU), the slowest rank's time is used and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "phase-space cell updates/s per step (FP32+MLP vs FP64 GPU) and % HBM roofline"
UNIT = "cell-updates/s"

from paper_2109_06743_gb300.workloads import NAMED as WORKLOADS  # noqa: E402
from paper_2109_06743_gb300.workloads import TRAIN_FROM, initial_state, initial_yee, x_line  # noqa: E402
from paper_2109_06743_gb300.workloads import named as make_cfg  # noqa: E402


def pin_host_to_gpu(device_index):
    """Run this process on the host cores local to the GPU (its PCI device's
    local_cpulist in sysfs), so that the pinned host buffers of the
    end-to-end leg are first touched, and placed, in the GPU's NUMA node.
    Returns the core list, or None where sysfs does not say."""
    import torch
    try:
        p = torch.cuda.get_device_properties(device_index)
        bdf = "%04x:%02x:%02x.0" % (getattr(p, "pci_domain_id", 0), p.pci_bus_id, p.pci_device_id)
        with open("/sys/bus/pci/devices/%s/local_cpulist" % bdf) as fh:
            spec = fh.read().strip()
        cpus = set()
        for part in spec.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        if not cpus or len(cpus) >= (os.cpu_count() or 0):
            return None
        os.sched_setaffinity(0, cpus)
        return spec
    except Exception:
        return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# FP32-pipe operations (add, multiply or fused multiply-add: one each) per
# velocity cell of one evaluation in the double-float Newton fit: moments of
# degree <= 2 (two double-float products for the recurrence, three
# compensated accumulations, the index step), plus the FP32 sums of degree
# <= 4 when the Jacobian is formed in the same pass, counted operation by
# operation.
OPS_MOMENT_EVAL = 46
OPS_GRAM_EVAL = 7
# DRAM bytes per cell of one fit launch (one species), by velocity grid, from
# the ncu captures of the warm-started 256 x 128 runs (32768 cells: targets,
# coefficients, status and the kernel's local memory): newton_kernel<16, 0>
# on the Harris sheet 11.37 MB read + 20.49 MB written, newton_kernel<12, 1>
# on the asymmetric sheet 12.54 + 49.85 MB; None for grids not captured.
NEWTON_DRAM_BYTES_PER_CELL = {16: (11.365e6 + 20.491e6) / 32768, 12: (12.545e6 + 49.848e6) / 32768}


def alu_peak_tops():
    """FP32-pipe peak from the unit counts and clock: 152 SMs x 128 FP32
    lanes x the maximum SM clock (MEASURED_PEAKS.json, else 2070 MHz)."""
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            mhz = float(json.load(fh).get("sm_max_mhz", mhz))
    return 152 * 128 * mhz * 1e6 / 1e12


def newton_roofline(cfg, stats, fit_ms, launches):
    """ALU roofline of the Newton fit kernel over the timed region: the
    algorithmic FP32-pipe operations (device counters of the evaluations x
    velocity cells x operations per cell) over the kernel's CUDA-event time."""
    if not fit_ms:
        return None
    n3 = cfg.species[0].nv[0] ** 3
    ops = (OPS_MOMENT_EVAL * (stats[4] + stats[6]) + OPS_GRAM_EVAL * (stats[5] + stats[7])) * n3
    achieved = ops / (fit_ms / 1e3) / 1e12
    peak = alu_peak_tops()
    per_cell = NEWTON_DRAM_BYTES_PER_CELL.get(cfg.species[0].nv[0])
    traffic = None if per_cell is None else per_cell * cfg.ncell
    return {"kernel": "fit_solve (newton_kernel)", "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "Tops/s (FP32 pipe)", "frac": achieved / peak, "traffic": traffic,
            "peak_kind": "derived: 152 SMs x 128 FP32 lanes x max SM clock",
            "ops_per_launch": ops / max(1, launches),
            "evaluations": {"moments": stats[4], "gram": stats[5], "slow": stats[6], "precise_steps": stats[7]}}


def slowest(seconds, dist=None, device="cpu"):
    """The replicas' wall time: the largest value over all ranks (identity
    without a process group)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, steps, world, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (replicas: every rank processes the same workload)."""
    return units_per_rank * steps * world / seconds


def accuracy_case(name):
    """The FP32 run checked against the FP64 oracle: for the Harris sheet a
    64 x 32 subdomain with the workload's dx, dv and dt (2 steps); for the
    asymmetric sheet a downscaled run of the sheet, 64 x 32 cells over
    6.4 x 3.2 (half the workload's resolution, five cells across the sheet
    half-width) with the workload's velocity grid (4 steps)."""
    from paper_2109_06743_gb300 import workloads as W
    kind, nx, ny, nv, lx, ly = WORKLOADS[name]
    if kind == "asym":
        return W.asym_sheet(nx=64, ny=32, nv=nv, lx=6.4, ly=3.2, precision=32), 4
    return make_cfg(name, precision=32, sub=(64, 32)), 2


def subdomain_accuracy(name, mlp_w, device):
    """Accuracy of the timed form (FP32 f, warm-started fits) against the
    FP64 oracle on the workload's accuracy case: relative L1 error of f, the
    largest moment error relative to the moment's absolute scale
    sum |v^alpha| f dv^3, both total-energy drifts, the energy partition
    (kinetic+thermal per species, electric, magnetic) on both sides, and the
    reconnected flux on the X line; the oracle's own time is the CPU
    baseline (one host core)."""
    import numpy as np

    import oracle
    from oracle.step import OracleState
    from paper_2109_06743_gb300 import abi
    from paper_2109_06743_gb300.driver import Simulation
    oracle.build()
    cfg, steps = accuracy_case(name)
    nv = cfg.species[0].nv[0]
    f64 = initial_state(cfg, np.float64)
    f32 = [x.astype(np.float32) for x in f64]
    yee = initial_yee(cfg)
    yl = x_line(cfg)
    sim = Simulation(cfg, f32, None, yee, device=device)
    if mlp_w is not None:
        abi.mlp_set_weights(sim.ctx, mlp_w)
    ost = OracleState(cfg, [x.astype(np.float64) for x in f32], None, yee)
    e0_gpu, e0_or = sim.total_energy(), ost.total_energy()
    part0 = ost.energies()
    psi0 = ost.reconnected_flux(yl)
    t0 = time.perf_counter()
    for _ in range(steps):
        ost.step(cfg.dt)
    t_or = time.perf_counter() - t0
    for _ in range(steps):
        sim.step(use_mlp=mlp_w is not None)
    l1, mom = [], []
    for k in range(len(cfg.species)):
        a, b = sim.f_host(k), ost.f[k]
        l1.append(float(np.abs(a - b).sum() / np.abs(b).sum()))
        mg = sim.mom_t[k].cpu().numpy()
        mo = oracle.moments(ost.f[k], ost.g, ost.sps[k])
        # scale of moment alpha: sum |v^alpha| f dv^3 (odd moments vanish by symmetry)
        sp = cfg.species[k]
        vs = [np.abs(sp.vcentres(ax)) for ax in range(3)]
        fb = ost.f[k].reshape(cfg.ncell, sp.nv[2], sp.nv[1], sp.nv[0])
        dv3 = float(np.prod([(sp.vmax[ax] - sp.vmin[ax]) / sp.nv[ax] for ax in range(3)]))
        powers = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1),
                  (0, 0, 2), (3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1),
                  (0, 1, 2), (0, 0, 3)]
        scale = np.stack([np.einsum("czyx,x,y,z->c", fb, vs[0] ** a, vs[1] ** b, vs[2] ** c_) * dv3
                          for a, b, c_ in powers], axis=1) + 1e-300
        mom.append(float((np.abs(mg - mo) / scale).max()))
    e1_gpu, e1_or = sim.total_energy(), ost.total_energy()
    psi_gpu, psi_or = sim.reconnected_flux(yl), ost.reconnected_flux(yl)

    def channels(e):
        kin, ee, eb = e
        return [float(x) for x in list(kin) + [ee, eb]]
    p_gpu, p_or, p0 = channels(sim.energies()), channels(ost.energies()), channels(part0)
    sim.close()
    cells = cfg.phase_cells() * steps
    what = ("%dx%d x %d^3 per species, 2 species, %d steps, " % (cfg.nx, cfg.ny, nv, steps)
            + ("downscaled whole sheet (dx %.2f), velocity grid and dt rule of the workload" % cfg.dx
               if cfg.kind == "asym" else "dx, dv, dt of the workload"))
    return {"run": what,
            "f_l1_rel_error": max(l1), "moment_max_rel_error": max(mom),
            "energy_drift_gpu": (e1_gpu - e0_gpu) / e0_gpu, "energy_drift_oracle": (e1_or - e0_or) / e0_or,
            "energy_gpu_vs_oracle": (e1_gpu - e1_or) / e1_or,
            "energy_partition": {"channels": ["kinetic+thermal e", "kinetic+thermal i", "electric", "magnetic"],
                                 "fraction_gpu": [x / sum(p_gpu) for x in p_gpu],
                                 "fraction_oracle": [x / sum(p_or) for x in p_or],
                                 "change_gpu": [a - b for a, b in zip(p_gpu, p0)],
                                 "change_oracle": [a - b for a, b in zip(p_or, p0)],
                                 "max_channel_error_rel_total": max(abs(a - b) for a, b in zip(p_gpu, p_or))
                                 / sum(p_or)},
            "x_line_y": yl,
            "reconnected_flux_rel_error": abs(psi_gpu - psi_or) / psi_or,
            "reconnection_rate_gpu": (psi_gpu - psi0) / (steps * cfg.dt),
            "reconnection_rate_oracle": (psi_or - psi0) / (steps * cfg.dt)}, {
        "value": cells / t_or, "unit": UNIT, "cores": 1, "kind": "oracle",
        "sample": "%d oracle steps of the %s sheet, %dx%d x %d^3 (2 species, %d cells), FP64, one host core, %.1f s" % (
            steps, cfg.kind, cfg.nx, cfg.ny, nv, cfg.phase_cells(), t_or)}


def cpu_baseline(name, steps=1, sample=(32, 16)):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    the central sample[0] x sample[1] spatial subdomain with the workload's
    dx, dv and dt (both species), one Algorithm 1 step per timed step,
    single-threaded."""
    import numpy as np

    from oracle.step import OracleState
    cfg = make_cfg(name, precision=64, sub=sample)
    st = OracleState(cfg, initial_state(cfg, np.float64), None, initial_yee(cfg))
    t0 = time.perf_counter()
    for _ in range(steps):
        st.step(cfg.dt)
    el = time.perf_counter() - t0
    cells = cfg.phase_cells() * steps
    nv = cfg.species[0].nv[0]
    return {"value": cells / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d oracle step(s) of the %s sheet on a %dx%d x %d^3 subdomain (2 species, %d cells, "
                      "same dx, dv, dt as the workload), FP64, one host core, %.1f s" % (
                          steps, cfg.kind, cfg.nx, cfg.ny, nv, cfg.phase_cells(), el)}


LANDAU = "landau_64_v32"


def run_landau(args, rank):
    """Config 1's line: 1D1V linear Landau damping (Sec. 3.1), 64 x 32 cells,
    FP64, the whole Algorithm 1 step (Strang x/2, v, x/2, Poisson, fluid,
    fit) per step. The workload fits in L2 and its kernels take microseconds,
    so the K timed steps are captured once in a CUDA graph and replayed (the
    step-by-step launch from Python is reported beside it); the oracle is
    timed on the same steps of the same workload and compared with it."""
    import numpy as np
    import torch

    import oracle
    from oracle.step import OracleState
    from paper_2109_06743_gb300 import abi
    from paper_2109_06743_gb300 import build as B
    from paper_2109_06743_gb300 import workloads as W
    from paper_2109_06743_gb300.driver import Simulation
    if rank != 0:
        return 0
    B.build()
    abi.lib()
    oracle.build()
    cfg = W.landau()
    f0 = W.landau_state(cfg)
    sim = Simulation(cfg, f0, stream=torch.cuda.Stream())
    stream = sim.stream
    cells = cfg.phase_cells()
    for _ in range(args.warmup):
        sim.step()
    torch.cuda.synchronize()
    # launched step by step from Python (host-bound: ~16 launches per step)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        sim.step()
    b.record(stream)
    torch.cuda.synchronize()
    eager = a.elapsed_time(b) / 1e3
    # the timed form: the K steps captured once in a CUDA graph and replayed
    l0 = abi.vl_launch_count()
    graph = sim.graph(args.steps)
    launches = abi.vl_launch_count() - l0
    with torch.cuda.stream(stream):  # a graph replays on the current stream
        graph.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    with torch.cuda.stream(stream):
        a.record(stream)
        graph.replay()
        b.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    el = a.elapsed_time(b) / 1e3
    # end to end: f from and back to pinned host memory every step
    host = [torch.empty(f.shape, dtype=f.dtype, pin_memory=True) for f in sim.f]
    for h, f in zip(host, sim.f):
        h.copy_(f)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.host_streams_after(e0)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            sim.step_through_host(host)
        sim.wait_host()
    e1.record(stream)
    torch.cuda.synchronize()
    et = e0.elapsed_time(e1) / 1e3
    nbytes = sum(f.numel() * f.element_size() for f in sim.f)
    sim.close()
    # the same number of steps of the oracle from the same f, against a
    # fresh GPU run of those steps
    g = Simulation(cfg, f0)
    ost = OracleState(cfg, f0)
    E0g, E0o = g.total_energy(), ost.total_energy()
    n = args.warmup + args.steps
    t0 = time.perf_counter()
    for _ in range(n):
        ost.step(cfg.dt)
    t_or = time.perf_counter() - t0
    for _ in range(n):
        g.step()
    diff = float(np.abs(g.f_host(0) - ost.f[0]).max() / ost.f[0].max())
    acc = {"steps": n, "f_max_rel_error": diff,
           "mass_rel_change_gpu": float(g.f_host(0).sum() / f0[0].sum() - 1.0),
           "energy_drift_gpu": (g.total_energy() - E0g) / E0g, "energy_drift_oracle": (ost.total_energy() - E0o) / E0o}
    g.close()
    peak, peak_kind = peaks()
    # algorithmic bytes per step: f read and written by the two half sweeps in
    # x, the velocity sweep and the exchange (8 B each way in FP64)
    step_bytes = 4 * 16 * cells
    line = {"metric": METRIC, "value": cells * args.steps / el, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": LANDAU, "grid": [cfg.nx, cfg.species[0].nv[0]], "species": 1,
                       "phase_cells_per_gpu": cells, "precision": "f64", "splitting": "strang x/2, v, x/2",
                       "l2": "the workload fits in L2 (%d KB of f): launch-latency bound" % (8 * cells // 1024),
                       "parallelism": "single"},
            "roofline": {"kernel": "whole step (L2-resident)", "bound": "hbm",
                         "achieved": step_bytes / (el / args.steps) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": step_bytes / (el / args.steps) / 1e9 / peak, "traffic": None,
                         "peak_kind": peak_kind, "algorithmic_bytes_per_launch": step_bytes},
            "accuracy_vs_fp64_oracle": acc,
            "cpu_baseline": {"value": cells * n / t_or, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "the whole workload, %d oracle steps, FP64, one host core, %.2f s" % (n, t_or)},
            "e2e": {"value": cells * args.steps / et, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "steps": args.steps},
            "gpu_launches": launches, "clocks": clk,
            "launched_from_python": {"value": cells * args.steps / eager, "unit": UNIT,
                                     "ms_per_step": 1e3 * eager / args.steps}}
    print(json.dumps(line))
    return 0


def _oracle_sample(name, sample, steps):
    """One process of the all-cores oracle figure: the sample run, timed."""
    import numpy as np

    from oracle.step import OracleState
    cfg = make_cfg(name, precision=64, sub=sample)
    st = OracleState(cfg, initial_state(cfg, np.float64), None, initial_yee(cfg))
    t0 = time.perf_counter()
    for _ in range(steps):
        st.step(cfg.dt)
    return cfg.phase_cells() * steps, time.perf_counter() - t0


def cpu_all_cores(name, sample=(32, 16), steps=1):
    """The oracle as it stands on every host core: one independent sample run
    per core, each in its own spawned process (the oracle itself is
    single-threaded); aggregate rate = all processes' cells over the slowest
    process's time."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import platform

    import oracle
    oracle.build()
    n = os.cpu_count() or 1
    with cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_sample, [name] * n, [sample] * n, [steps] * n))
    cells = sum(c for c, _ in res)
    slow = max(t for _, t in res)
    return {"value": cells / slow, "unit": UNIT, "cores": n, "kind": "oracle", "machine": platform.machine(),
            "sample": "%d processes, each %d oracle step(s) of the %dx%d subdomain (same dx, dv, dt as the "
                      "workload), FP64; slowest process %.1f s" % (n, steps, sample[0], sample[1], slow)}


def run_reference(args, rank):
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; warm-up steps are not needed
    if args.workload == LANDAU:
        from oracle.step import OracleState
        from paper_2109_06743_gb300 import workloads as W
        cfg = W.landau()
        st = OracleState(cfg, W.landau_state(cfg))
        t0 = time.perf_counter()
        for _ in range(args.steps):
            st.step(cfg.dt)
        el = time.perf_counter() - t0
        cb = {"value": cfg.phase_cells() * args.steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": "the whole workload, %d oracle steps, FP64, one host core, %.2f s" % (args.steps, el)}
    else:
        cb = cpu_baseline(args.workload, steps=args.steps, sample=(16, 8))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "ms_per_step": None,
            "config": {"workload": args.workload + (" (the whole workload)" if args.workload == LANDAU
                                                    else " (oracle sample: 16x8 spatial subdomain)")},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="harris_512x256_v16", choices=sorted(WORKLOADS) + [LANDAU])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2, help="steps of the FP64 form timed for comparison")
    ap.add_argument("--no-mlp", action="store_true", help="cold-started fits only (no warm-start network)")
    ap.add_argument("--train-from", default=None, choices=sorted(WORKLOADS),
                    help="workload whose fits train the warm-start network (default: the same velocity grid)")
    ap.add_argument("--harvest-steps", type=int, default=24, help="cold-started steps harvested for training")
    ap.add_argument("--no-all-cores", action="store_true", help="skip the all-cores oracle figure")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == LANDAU:
        return run_landau(args, rank)

    import numpy as np
    import torch

    from paper_2109_06743_gb300 import abi
    from paper_2109_06743_gb300 import build as B
    from paper_2109_06743_gb300.driver import Simulation
    from paper_2109_06743_gb300.warmstart import train_warm_start

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    abi.lib()

    device = "cuda:%d" % local
    affinity = pin_host_to_gpu(local)
    train_from = args.train_from or TRAIN_FROM[args.workload]
    mlp_w, mlp_info = (None, None) if args.no_mlp else train_warm_start(train_from, device,
                                                                         harvest_steps=args.harvest_steps)
    use_mlp = mlp_w is not None
    cfg = make_cfg(args.workload, precision=32)
    f0 = initial_state(cfg, np.float32)
    sim = Simulation(cfg, f0, None, initial_yee(cfg), device=device)
    if use_mlp:
        abi.mlp_set_weights(sim.ctx, mlp_w)
    stream = sim.stream
    cells = cfg.phase_cells()

    def barrier_sync():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        sim.step(use_mlp=use_mlp)
    abi.vl_reset_stats(sim.ctx, stream)
    barrier_sync()

    # ---- timed region: K steps, CUDA events on the solver's stream ----------
    phase_ms = {}
    pending = []
    cur = {"label": None, "ev": None}

    def mark(label):
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        if cur["label"] is not None:
            pending.append((cur["label"], cur["ev"], ev))
        cur["label"], cur["ev"] = label, ev

    clocks = ClockSampler(local)
    clocks.start()
    launches0 = abi.vl_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        sim.step(use_mlp=use_mlp, mark=mark)
    t_end.record(stream)
    barrier_sync()
    launches = abi.vl_launch_count() - launches0
    clk = clocks.stop()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    count = {}
    for label, e0, e1 in pending:
        phase_ms[label] = phase_ms.get(label, 0.0) + e0.elapsed_time(e1)
        count[label] = count.get(label, 0) + 1
    stats = abi.vl_read_stats(sim.ctx, stream)
    if stats[8]:
        raise RuntimeError("%d tile copies of the fused sweep ran out of time: the timed steps are invalid" % stats[8])
    elapsed = slowest(elapsed, dist, device)
    value = job_rate(cells, args.steps, world, elapsed)

    # ---- roofline of the dominant kernel --------------------------------------
    peak, peak_kind = peaks()
    per_launch_cells = cells // len(cfg.species)  # one species per launch
    hbm_phases = {"xy_sweep": 8, "x_sweep": 8, "y_sweep": 8, "v_pass": 8, "fit_exchange": 8}
    dom = max(phase_ms, key=lambda k: phase_ms[k])
    rows = {}
    for ph, b in hbm_phases.items():
        if ph in phase_ms:
            avg_s = phase_ms[ph] / count[ph] / 1e3
            rows[ph] = {"ms_per_launch": avg_s * 1e3, "GBps": b * per_launch_cells / avg_s / 1e9,
                        "frac_of_%s_hbm" % peak_kind: b * per_launch_cells / avg_s / 1e9 / peak}
    newton = newton_roofline(cfg, stats, phase_ms.get("fit_solve"), count.get("fit_solve", 1))
    if dom in hbm_phases:
        roof = {"kernel": dom, "bound": "hbm", "achieved": rows[dom]["GBps"], "peak": peak, "unit": "GB/s",
                "frac": rows[dom]["GBps"] / peak, "traffic": None, "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": 8 * per_launch_cells}
    else:
        roof = newton

    # ---- the same steps with the cold-started fit (no network) ----------------
    cold = None
    if use_mlp:
        kc = max(1, min(args.steps, 5))
        abi.vl_reset_stats(sim.ctx, stream)
        barrier_sync()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(kc):
            sim.step(use_mlp=False)
        c1.record(stream)
        barrier_sync()
        tc_ = c0.elapsed_time(c1) / 1e3
        cst = abi.vl_read_stats(sim.ctx, stream)
        nfit = 2 * cfg.ncell * len(cfg.species)
        cold = {"value": cells * kc / tc_, "unit": UNIT, "ms_per_step": 1e3 * tc_ / kc, "steps": kc,
                "newton_iterations_per_fit": cst[0] / (nfit * kc), "newton_fallbacks_per_fit": cst[1] / (nfit * kc)}

    # ---- end to end through the public API with host buffers ------------------
    e2e = None
    if not args.no_e2e:
        host = [torch.empty(f.shape, dtype=f.dtype, pin_memory=True) for f in sim.f]
        for h, f in zip(host, sim.f):
            h.copy_(f)
        barrier_sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ksteps = max(1, min(args.steps, 10))
        e0.record(stream)
        sim.host_streams_after(e0)
        with torch.cuda.stream(stream):
            for _ in range(ksteps):
                sim.step_through_host(host, use_mlp=use_mlp)
            sim.wait_host()
        e1.record(stream)
        barrier_sync()
        et = slowest(e0.elapsed_time(e1) / 1e3, dist, device)
        nbytes = sum(f.numel() * f.element_size() for f in sim.f)
        e2e = {"value": job_rate(cells, ksteps, world, et), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": ksteps}

    nfits = max(1, 2 * cfg.ncell * len(cfg.species) * args.steps)
    fit_iters = stats[0] / nfits
    if use_mlp:
        mlp_info.update({"newton_iterations_per_fit": fit_iters, "newton_fallbacks_per_fit": stats[1] / nfits,
                         "cold_start": cold,
                         "applied_to": args.workload + " (%d^3 velocity cells per species)" % cfg.species[0].nv[0]})
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # ---- the plain FP64 GPU form of the same workload -------------------------
    fp64 = None
    if args.fp64_steps > 0:
        cfg64 = make_cfg(args.workload, precision=64)
        s64 = Simulation(cfg64, initial_state(cfg64, np.float64), None, initial_yee(cfg64),
                         device="cuda:%d" % local)
        for _ in range(3):
            s64.step()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s64.stream)
        for _ in range(args.fp64_steps):
            s64.step()
        b.record(s64.stream)
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b) / 1e3
        fp64 = {"value": cells * args.fp64_steps / t64, "unit": UNIT, "ms_per_step": 1e3 * t64 / args.fp64_steps,
                "steps": args.fp64_steps, "note": "same workload with FP64 f and sweeps, single GPU"}
        s64.close()

    if rank != 0:
        return 0
    acc, cb = (None, None) if args.no_cpu else subdomain_accuracy(args.workload, mlp_w, device)
    if cb is not None and not args.no_all_cores:
        cb["all_cores"] = cpu_all_cores(args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "grid": [cfg.nx, cfg.ny], "nv": cfg.species[0].nv[0],
                   "species": len(cfg.species), "phase_cells_per_gpu": cells,
                   "precision": "f32 f, sweeps and fluid right-hand side; f64 moment sums, fluid state, fields; "
                                "double-float Newton fit" + ("; BF16 warm-start network" if use_mlp else ""),
                   "splitting": "lie x,y,v; 5-shear Boris velocity map", "l2": "inputs larger than L2 (f %.1f GB)" % (
                       sum(cfg.ncell * s.vblock for s in cfg.species) * 4 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single", "host_cores": affinity},
        "roofline": roof,
        "phases_ms_per_step": {k: v / args.steps for k, v in sorted(phase_ms.items())},
        "hbm_phases": rows,
        "newton_iterations_per_fit": fit_iters, "newton_fallbacks": stats[1], "clipped_cells": stats[2],
        "mlp": mlp_info, "accuracy_vs_fp64_oracle": acc,
        "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches, "clocks": clk, "fp64_form": fp64,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
