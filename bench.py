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
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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


# Work of the Newton fits per velocity cell and evaluation of a discrete
# Maxwellian, in operations (add, multiply or fused multiply-add: one each).
# The method's own work (Sec. 2.2's discrete fit): the ten moment sums of
# degree <= 2 per evaluation, and 25 more sums (degree 3 and 4, the entries
# of the Gram matrix beyond the moments) when the Jacobian is formed.
METHOD_OPS_MOMENT = 10
METHOD_OPS_GRAM = 25
# What the double-float kernels issue on the FP32 (FMA) pipe for the same
# work, counted operation by operation: two double-float products for the
# recurrence, three compensated accumulations and the index step -- 30 in
# the edge-start pass of the common kernel, whose accumulations order their
# operands on the ALU pipe (7 more operations there), add by Fast2Sum and
# take their weighted terms as chained products, and whose products skip
# the renormalisation (the ratio's always, the value's without the
# Jacobian; counted here as in the moment-only pass), 43 in the centre-out
# pass of the wide kernel (TwoSum, the ratio unnormalised) -- plus the FP32
# sums of degree <= 4 and the value's renormalisation when the Jacobian is
# formed in the same pass (9).
ISSUED_OPS_MOMENT_EDGE = 30
ISSUED_ALU_OPS_MOMENT_EDGE = 7
ISSUED_OPS_MOMENT_CENTRE = 43
ISSUED_OPS_GRAM_DF = 9
# What the FP64 kernel issues on the FP64 pipe: the two products of the
# recurrence and three accumulations (5), plus two accumulations with the
# Gram sums (2).
ISSUED_OPS_MOMENT_64 = 5
ISSUED_OPS_GRAM_64 = 2
# DRAM bytes per cell of one fit launch (one species), by kernel (FP64 or
# not) and velocity grid, from ncu captures of the current kernels on the
# 256 x 128 Harris sheet (dram__bytes_read.sum + dram__bytes_write.sum over
# 32768 cells; scaled by the cell count, as the traffic is per cell): the
# double-float kernel warm-started, 36.66 MB (targets, coefficients, status,
# predictions and its local memory), the FP64 kernel cold-started, 8.20 MB
# (its coefficient writes stay in L2 during the launch). A grid not captured
# gives None.
# timed runs of the end-to-end leg (the fastest is reported, all are listed)
E2E_REPS = 8
NEWTON_DRAM_BYTES_PER_CELL = {(False, 16): 36.659200e6 / 32768, (True, 16): 8.204032e6 / 32768}
# Bytes a fit launch must move per cell: the 20 raw moments (read), the fluid
# state (10 doubles read and written), both Maxwellians' 16 coefficients
# (written), the status pair and, warm-started, the network's 20 predictions.
NEWTON_ALGORITHMIC_BYTES_PER_CELL = 20 * 8 + 2 * 10 * 8 + 2 * 16 * 8 + 2 * 4
NEWTON_WARM_BYTES_PER_CELL = 20 * 4


def measured_alu_peaks(device):
    """FMA operations per second of this GPU in FP32 and FP64, measured by
    the library's probe kernel (vl_fma_peak: independent FMA chains timed
    with CUDA events; no device setting is changed)."""
    import torch

    from paper_2109_06743_gb300 import abi
    sink = torch.zeros(1, dtype=torch.float64, device=device)
    p32 = abi.vl_fma_peak(32, sink)
    p64 = abi.vl_fma_peak(64, sink)
    return {"fp32_tops": p32 / 1e12, "fp64_tops": p64 / 1e12,
            "how": "vl_fma_peak: 8 independent FMA chains per thread, 8 x 256-thread blocks per SM, CUDA events, "
                   "FMA counted as one operation"}


def newton_roofline(cfg, stats, fit_ms, launches, alu, fp64=False):
    """ALU roofline of the Newton fit kernel over the timed region. achieved
    = the method's operations (device counters of the evaluations x
    velocity cells x METHOD_OPS_*) over the kernel's CUDA-event time; peak =
    the measured FMA rate of the pipe the kernel computes on (FP32 for the
    double-float fit, FP64 for the FP64 fit). The operations the kernel
    actually issues for that work are reported beside it."""
    if not fit_ms:
        return None
    n3 = cfg.species[0].nv[0] ** 3
    secs = fit_ms / 1e3
    if fp64:
        em, eg = stats[10], stats[11]
        issued = (ISSUED_OPS_MOMENT_64 * em + ISSUED_OPS_GRAM_64 * eg) * n3
        peak = alu["fp64_tops"]
        kernel, pipe = "fit_solve (newton64_kernel, FP64)", "FP64"
        evals = {"moments": em, "gram": eg}
    else:
        em, eg = stats[4] + stats[6], stats[5] + stats[7]
        # the wide kernel takes whole species: its share of the fits
        w = min(1.0, stats[9] / max(1, 2 * cfg.ncell * launches))
        issued = ((ISSUED_OPS_MOMENT_EDGE * (1 - w) + ISSUED_OPS_MOMENT_CENTRE * w) * em + ISSUED_OPS_GRAM_DF * eg) * n3
        issued_alu = ISSUED_ALU_OPS_MOMENT_EDGE * (1 - w) * em * n3
        peak = alu["fp32_tops"]
        kernel, pipe = "fit_solve (newton_kernel, double-float on the FP32 pipe)", "FP32"
        evals = {"moments": stats[4], "gram": stats[5], "slow": stats[6], "precise_steps": stats[7],
                 "wide_kernel_fits": stats[9]}
    method = (METHOD_OPS_MOMENT * em + METHOD_OPS_GRAM * eg) * n3
    achieved = method / secs / 1e12
    per_cell = NEWTON_DRAM_BYTES_PER_CELL.get((fp64, cfg.species[0].nv[0]))
    alg = NEWTON_ALGORITHMIC_BYTES_PER_CELL + (0 if fp64 else NEWTON_WARM_BYTES_PER_CELL)
    out = {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s (%s pipe)" % pipe,
           "frac": achieved / peak, "traffic": None if per_cell is None else per_cell * cfg.ncell,
           "algorithmic_bytes_per_launch": alg * cfg.ncell,
           "peak_kind": "measured (vl_fma_peak)",
           "method_ops_per_launch": method / max(1, launches), "method_frac": achieved / peak,
           "issued_ops_per_launch": issued / max(1, launches), "issued_frac": issued / secs / 1e12 / peak,
           "evaluations": evals}
    if not fp64:
        out["method_vs_fp64_peak"] = achieved / alu["fp64_tops"]
        out["issued_alu_ops_per_launch"] = issued_alu / max(1, launches)
    return out


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
    return {"value": cells / el, "unit": UNIT, "cores": 1, "kind": "oracle", "sample_ms_per_step": 1e3 * el / steps,
            "sample": "%d oracle step(s) of the %s sheet on a %dx%d x %d^3 subdomain (2 species, %d cells, "
                      "same dx, dv, dt as the workload), FP64, one host core, %.1f s" % (
                          steps, cfg.kind, cfg.nx, cfg.ny, nv, cfg.phase_cells(), el)}


LANDAU = "landau_64_v32"


def landau_block(steps, warmup):
    """Config 1's measurement: 1D1V linear Landau damping (Sec. 3.1), 64 x 32
    cells, FP64, the whole Algorithm 1 step (Strang x/2, v, x/2, Poisson,
    fluid, fit) per step. The workload fits in L2 and its kernels take
    microseconds, so the K timed steps are captured once in a CUDA graph and
    replayed (the step-by-step launch from Python is reported beside it);
    the oracle is timed on the same steps of the same workload and compared
    with it. Returns the fields of a bench line."""
    import numpy as np
    import torch

    import oracle
    from oracle.step import OracleState
    from paper_2109_06743_gb300 import abi
    from paper_2109_06743_gb300 import workloads as W
    from paper_2109_06743_gb300.driver import Simulation
    oracle.build()
    cfg = W.landau()
    f0 = W.landau_state(cfg)
    sim = Simulation(cfg, f0, stream=torch.cuda.Stream())
    stream = sim.stream
    cells = cfg.phase_cells()
    for _ in range(warmup):
        sim.step()
    torch.cuda.synchronize()
    # launched step by step from Python (host-bound: ~16 launches per step)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        sim.step()
    b.record(stream)
    torch.cuda.synchronize()
    eager = a.elapsed_time(b) / 1e3
    # the timed form: the K steps captured once in a CUDA graph and replayed
    l0 = abi.vl_launch_count()
    graph = sim.graph(steps)
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
        for _ in range(steps):
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
    n = warmup + steps
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
    return {"metric": METRIC, "value": cells * steps / el, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": LANDAU, "grid": [cfg.nx, cfg.species[0].nv[0]], "species": 1,
                       "phase_cells_per_gpu": cells, "precision": "f64", "splitting": "strang x/2, v, x/2",
                       "l2": "the workload fits in L2 (%d KB of f): launch-latency bound" % (8 * cells // 1024),
                       "parallelism": "single"},
            "roofline": {"kernel": "whole step (L2-resident)", "bound": "hbm",
                         "achieved": step_bytes / (el / steps) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": step_bytes / (el / steps) / 1e9 / peak, "traffic": None,
                         "peak_kind": peak_kind, "algorithmic_bytes_per_launch": step_bytes},
            "accuracy_vs_fp64_oracle": acc,
            "cpu_baseline": {"value": cells * n / t_or, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "the whole workload, %d oracle steps, FP64, one host core, %.2f s" % (n, t_or)},
            "e2e": {"value": cells * steps / et, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "steps": steps},
            "gpu_launches": launches, "clocks": clk,
            "launched_from_python": {"value": cells * steps / eager, "unit": UNIT,
                                     "ms_per_step": 1e3 * eager / steps}}


def run_landau(args, rank):
    """The Landau workload as the bench line itself (--workload landau_64_v32)."""
    from paper_2109_06743_gb300 import abi
    from paper_2109_06743_gb300 import build as B
    if rank != 0:
        return 0
    B.build()
    abi.lib()
    print(json.dumps(landau_block(args.steps, args.warmup)))
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
              "sample_ms_per_step": 1e3 * el / args.steps,
              "sample": "the whole workload, %d oracle steps, FP64, one host core, %.2f s" % (args.steps, el)}
    else:
        cb = cpu_baseline(args.workload, steps=args.steps, sample=(16, 8))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            # a step of the whole workload only where the oracle ran the whole workload
            "ms_per_step": cb["sample_ms_per_step"] if args.workload == LANDAU else None,
            "config": {"workload": args.workload + (" (the whole workload)" if args.workload == LANDAU
                                                    else " (oracle sample: 16x8 spatial subdomain)")},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def timed_steps(sim, steps, use_mlp):
    """K steps on the solver's stream, bracketed by CUDA events, with an event
    before every phase; returns (seconds, {phase: ms}, {phase: launches},
    kernels launched by the library)."""
    import torch

    from paper_2109_06743_gb300 import abi
    stream = sim.stream
    pending = []
    cur = {"label": None, "ev": None}

    def mark(label):
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        if cur["label"] is not None:
            pending.append((cur["label"], cur["ev"], ev))
        cur["label"], cur["ev"] = label, ev

    l0 = abi.vl_launch_count()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        sim.step(use_mlp=use_mlp, mark=mark)
    t1.record(stream)
    torch.cuda.synchronize()
    launches = abi.vl_launch_count() - l0
    phase_ms, count = {}, {}
    for label, e0, e1 in pending:
        phase_ms[label] = phase_ms.get(label, 0.0) + e0.elapsed_time(e1)
        count[label] = count.get(label, 0) + 1
    return t0.elapsed_time(t1) / 1e3, phase_ms, count, launches


def hbm_rows(phase_ms, count, per_launch_cells, bytes_per_cell=8):
    """HBM fraction of each memory-bound pass: algorithmic bytes (f read and
    written once) per launch over the phase's CUDA-event time per launch."""
    peak, peak_kind = peaks()
    rows = {}
    for ph in ("xy_sweep", "x_sweep", "y_sweep", "v_pass", "fit_exchange"):
        if ph in phase_ms:
            avg_s = phase_ms[ph] / count[ph] / 1e3
            gbs = bytes_per_cell * per_launch_cells / avg_s / 1e9
            rows[ph] = {"ms_per_launch": avg_s * 1e3, "GBps": gbs, "frac_of_%s_hbm" % peak_kind: gbs / peak}
    return rows


def host_link(host, dev, reps=3, both_only=False):
    """Pinned host <-> device copy rates with plain cudaMemcpyAsync (torch
    copy_ of pinned tensors, one stream per direction): host to device
    alone, device to host alone, and both at once; the roof of the
    end-to-end leg, which moves f both ways every step. both_only: only
    the rate each way with both directions at once (GB/s)."""
    import torch
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    nbytes = sum(h.numel() * h.element_size() for h in host)

    def run(h2d, d2h):
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(s1)
            s2.wait_event(e[0])
            if h2d:
                with torch.cuda.stream(s1):
                    for h, d in zip(host, dev):
                        d.copy_(h, non_blocking=True)
            if d2h:
                with torch.cuda.stream(s2):
                    for h, d in zip(host, dev):
                        h.copy_(d, non_blocking=True)
            e[1].record(s1)
            e[2].record(s2)
            s1.wait_event(e[2])
            e[3].record(s1)
            torch.cuda.synchronize()
            t = e[0].elapsed_time(e[3]) / 1e3
            best = t if best is None else min(best, t)
        return best

    if both_only:
        return nbytes / run(True, True) / 1e9
    t_h2d = run(True, False)
    t_d2h = run(False, True)
    t_both = run(True, True)
    return {"bytes_each_way": nbytes, "h2d_GBps": nbytes / t_h2d / 1e9, "d2h_GBps": nbytes / t_d2h / 1e9,
            "both_directions_GBps_each_way": nbytes / t_both / 1e9,
            "step_copy_ms_at_roof": 1e3 * t_both,
            "how": "torch copy_ between pinned host and device tensors (cudaMemcpyAsync), one stream per "
                   "direction, best of %d" % reps}


def measure_2d3v(name, device, alu, steps, warmup, e2e_steps, cold_steps, fp64_steps, accuracy, all_cores,
                 harvest_steps=24, train_from=None, no_mlp=False, dist=None, world=1, gpu_index=0,
                 transfer_from=None, transfer_samples=0, fused_xy=True):
    """One 2D3V workload: the FP32+MLP form timed over `steps` steps (CUDA
    events per phase, clocks sampled), its roofline, the same steps with
    cold-started fits, optionally the warm-start network trained on another
    velocity grid (transfer_from), the end-to-end leg with the host link's
    own copy rates, the plain FP64 form, and (rank 0) the accuracy against
    the FP64 oracle with the oracle's rates as CPU baseline."""
    import numpy as np
    import torch

    from paper_2109_06743_gb300 import abi
    from paper_2109_06743_gb300.driver import Simulation
    from paper_2109_06743_gb300.warmstart import train_warm_start
    rank = dist.get_rank() if dist else 0
    train_from = train_from or TRAIN_FROM[name]
    mlp_w, mlp_info = (None, None) if no_mlp else train_warm_start(train_from, device, harvest_steps=harvest_steps)
    use_mlp = mlp_w is not None
    cfg = make_cfg(name, precision=32)
    sim = Simulation(cfg, initial_state(cfg, np.float32), None, initial_yee(cfg), device=device, fused_xy=fused_xy)
    if use_mlp:
        abi.mlp_set_weights(sim.ctx, mlp_w)
    stream = sim.stream
    cells = cfg.phase_cells()
    nsp = len(cfg.species)

    def barrier_sync():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(warmup):
        sim.step(use_mlp=use_mlp)
    abi.vl_reset_stats(sim.ctx, stream)
    barrier_sync()

    # ---- timed region: K steps, CUDA events on the solver's stream ----------
    clocks = ClockSampler(gpu_index)
    clocks.start()
    elapsed, phase_ms, count, launches = timed_steps(sim, steps, use_mlp)
    barrier_sync()
    clk = clocks.stop()
    stats = abi.vl_read_stats(sim.ctx, stream)
    if stats[8]:
        raise RuntimeError("%d tile copies of the fused sweep ran out of time: the timed steps are invalid" % stats[8])
    abi.vl_sync_status(sim.ctx, stream)
    elapsed = slowest(elapsed, dist, device)
    value = job_rate(cells, steps, world, elapsed)

    # ---- roofline of the dominant kernel --------------------------------------
    peak, peak_kind = peaks()
    per_launch_cells = cells // nsp  # one species per launch
    rows = hbm_rows(phase_ms, count, per_launch_cells)
    dom = max(phase_ms, key=lambda k: phase_ms[k])
    newton = newton_roofline(cfg, stats, phase_ms.get("fit_solve"), count.get("fit_solve", 1), alu)
    if dom in rows:
        roof = {"kernel": dom, "bound": "hbm", "achieved": rows[dom]["GBps"], "peak": peak, "unit": "GB/s",
                "frac": rows[dom]["GBps"] / peak, "traffic": None, "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": 8 * per_launch_cells}
    else:
        roof = newton
    nfit = 2 * cfg.ncell * nsp

    # ---- the same steps with the cold-started fit (no network) ----------------
    cold = None
    if use_mlp and cold_steps > 0:
        abi.vl_reset_stats(sim.ctx, stream)
        barrier_sync()
        tc_, ph_c, cnt_c, _ = timed_steps(sim, cold_steps, False)
        cst = abi.vl_read_stats(sim.ctx, stream)
        cold = {"value": cells * cold_steps / tc_, "unit": UNIT, "ms_per_step": 1e3 * tc_ / cold_steps,
                "steps": cold_steps, "fit_solve_ms_per_step": ph_c.get("fit_solve", 0.0) / cold_steps,
                "newton_iterations_per_fit": cst[0] / (nfit * cold_steps),
                "newton_fallbacks_per_fit": cst[1] / (nfit * cold_steps)}

    # ---- the network trained on another velocity grid (transfer) ---------------
    transfer = None
    if use_mlp and transfer_from:
        tw, tinfo = train_warm_start(transfer_from, device, harvest_steps=max(1, transfer_samples // (
            4 * make_cfg(transfer_from).ncell)))
        abi.mlp_set_weights(sim.ctx, tw)
        abi.vl_reset_stats(sim.ctx, stream)
        barrier_sync()
        kt = max(1, cold_steps)
        tt, ph_t, _, _ = timed_steps(sim, kt, True)
        tst = abi.vl_read_stats(sim.ctx, stream)
        abi.mlp_set_weights(sim.ctx, mlp_w)
        tinfo.update({"applied_to": "%s (%d^3 velocity cells per species)" % (name, cfg.species[0].nv[0]),
                      "steps": kt, "ms_per_step": 1e3 * tt / kt,
                      "fit_solve_ms_per_step": ph_t.get("fit_solve", 0.0) / kt,
                      "newton_iterations_per_fit": tst[0] / (nfit * kt),
                      "newton_fallbacks_per_fit": tst[1] / (nfit * kt),
                      "fits_started_warm": tst[12] / (nfit * kt)})
        transfer = tinfo

    # ---- end to end through the public API with host buffers ------------------
    e2e = None
    if e2e_steps > 0:
        host = [torch.empty(f.shape, dtype=f.dtype, pin_memory=True) for f in sim.f]
        for h, f in zip(host, sim.f):
            h.copy_(f)
        # E2E_REPS timed runs of e2e_steps steps each (the first step of a run
        # also fills the copy pipeline); the fastest run is the
        # figure, as for the host link's own rates (the link and the host's
        # memory are shared with the node's other GPUs, whose traffic can slow
        # any number of runs), and every run is listed with the both-ways copy
        # rate of the same buffers measured right before it
        reps, link_before = [], []
        for _ in range(E2E_REPS):
            barrier_sync()
            link_before.append(host_link(host, sim.f_spare or sim.f, reps=1, both_only=True))
            barrier_sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.host_streams_after(e0)
            with torch.cuda.stream(stream):
                for _ in range(e2e_steps):
                    sim.step_through_host(host, use_mlp=use_mlp)
                sim.wait_host()
            e1.record(stream)
            barrier_sync()
            reps.append(slowest(e0.elapsed_time(e1) / 1e3, dist, device))
        et = min(reps)
        nbytes = sum(f.numel() * f.element_size() for f in sim.f)
        link = host_link(host, sim.f_spare or sim.f)
        e2e = {"value": job_rate(cells, e2e_steps, world, et), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": e2e_steps, "ms_per_step": 1e3 * et / e2e_steps,
               "runs_ms_per_step": [1e3 * t / e2e_steps for t in reps], "run_reported": "fastest of %d" % E2E_REPS,
               "runs_link_GBps_each_way_before": link_before,
               "host_link": link,
               "copy_bound_value": cells / (link["step_copy_ms_at_roof"] / 1e3)}
        del host

    fit_iters = stats[0] / max(1, nfit * steps)
    if use_mlp:
        mlp_info.update({"newton_iterations_per_fit": fit_iters, "newton_fallbacks_per_fit": stats[1] / (nfit * steps),
                         "fits_started_warm": stats[12] / (nfit * steps), "cold_start": cold,
                         "applied_to": name + " (%d^3 velocity cells per species)" % cfg.species[0].nv[0]})
        if transfer:
            mlp_info["transfer"] = transfer
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # ---- the plain FP64 GPU form of the same workload -------------------------
    fp64 = None
    if fp64_steps > 0:
        cfg64 = make_cfg(name, precision=64)
        s64 = Simulation(cfg64, initial_state(cfg64, np.float64), None, initial_yee(cfg64), device=device)
        for _ in range(2):
            s64.step()
        abi.vl_reset_stats(s64.ctx, s64.stream)
        torch.cuda.synchronize()
        t64, ph64, cnt64, _ = timed_steps(s64, fp64_steps, False)
        st64 = abi.vl_read_stats(s64.ctx, s64.stream)
        nf64 = 2 * cfg64.ncell * len(cfg64.species) * fp64_steps
        fp64 = {"value": cells * fp64_steps / t64, "unit": UNIT, "ms_per_step": 1e3 * t64 / fp64_steps,
                "steps": fp64_steps, "phases_ms_per_step": {k: v / fp64_steps for k, v in sorted(ph64.items())},
                "hbm_phases": hbm_rows(ph64, cnt64, per_launch_cells, 16),
                "newton_iterations_per_fit": st64[0] / nf64, "newton_fallbacks_per_fit": st64[1] / nf64,
                "fit_roofline": newton_roofline(cfg64, st64, ph64.get("fit_solve"), cnt64.get("fit_solve", 1), alu,
                                                fp64=True),
                "note": "same workload, FP64 f, sweeps, fluid and plain FP64 Newton fit, cold-started"}
        s64.close()
        del s64
        torch.cuda.empty_cache()

    acc, cb = (None, None)
    if rank == 0 and accuracy:
        acc, cb = subdomain_accuracy(name, mlp_w, device)
        if all_cores:
            cb["all_cores"] = cpu_all_cores(name)
    return {
        "value": value, "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * elapsed / steps,
        "config": {"workload": name, "grid": [cfg.nx, cfg.ny], "nv": cfg.species[0].nv[0], "species": nsp,
                   "phase_cells_per_gpu": cells,
                   "precision": "f32 f, sweeps and fluid right-hand side; f64 moment sums, fluid state, fields; "
                                "double-float Newton fit" + ("; BF16 warm-start network" if use_mlp else ""),
                   "splitting": "lie x,y,v; 5-shear Boris velocity map",
                   "spatial_sweeps": "fused x+y (pfc_advect_xy)" if fused_xy else "single-axis x then y (pfc_advect_x)",
                   "l2": "inputs larger than L2 (f %.1f GB)" % (
                       sum(cfg.ncell * s_.vblock for s_ in cfg.species) * 4 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof, "newton_roofline": newton,
        "phases_ms_per_step": {k: v / steps for k, v in sorted(phase_ms.items())},
        "hbm_phases": rows,
        "newton_iterations_per_fit": fit_iters, "newton_fallbacks": stats[1], "clipped_cells": stats[2],
        "mlp": mlp_info, "accuracy_vs_fp64_oracle": acc,
        "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches, "clocks": clk, "fp64_form": fp64}


def launch_fixed_cost(device, step_ms, per_launch_ms, reps=50):
    """What batching the species into one launch could save (the fused
    sweep's multi-species batching): the fixed cost of one per-species
    launch -- launch, per-CTA set-up, and a last partial wave -- measured as
    the whole duration of the same pass on a 16 x 16 window (the workload's
    dx, dv and dt), where one partial wave of persistent CTAs does all the
    work. CUDA events around each call (the velocity pass's call includes its
    shear set-up kernel); the bound is one such cost per pass and step for the
    second species, against the full step."""
    import numpy as np
    import torch

    from paper_2109_06743_gb300 import abi
    from paper_2109_06743_gb300.driver import Simulation
    cfg = make_cfg("harris_512x256_v16", precision=32, sub=(16, 16))
    sim = Simulation(cfg, initial_state(cfg, np.float32), None, initial_yee(cfg), device=device)
    st = sim.stream
    out = {"window": "16x16 x 16^3, one species, the workload's dx, dv and dt", "reps": reps}
    for name in ("xy_sweep", "v_pass"):
        evs = []
        with torch.cuda.stream(st):
            for r in range(reps + 3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                if name == "xy_sweep":
                    abi.pfc_advect_xy(sim.ctx, 0, cfg.dt, sim.f_spare[0], st)
                    sim.f[0], sim.f_spare[0] = sim.f_spare[0], sim.f[0]
                else:
                    abi.pfc_advect_v(sim.ctx, 0, cfg.dt, None, st)
                e1.record(st)
                if r >= 3:
                    evs.append((e0, e1))
        torch.cuda.synchronize()
        us = sorted(1e3 * a.elapsed_time(b) for a, b in evs)
        out[name + "_us"] = us[len(us) // 2]
        if per_launch_ms.get(name):
            out[name + "_full_size_ms_per_species"] = per_launch_ms[name]
    sim.close()
    out["batching_bound_pct_of_step"] = 100.0 * 1e-3 * (out["xy_sweep_us"] + out["v_pass_us"]) / step_ms
    return out


def shear_ablation(device, steps=100):
    """The velocity splitting read two ways (Sec. 2.1's backsubstitution):
    the exact five-shear factorisation of the Boris map against the plain
    three-shear split, on the Harris subdomain of the accuracy check (64 x 32
    x 16^3, the workload's dx, dv and dt), FP64, fitted, `steps` steps on the
    GPU: total-energy drift of each, and the difference of the two runs'
    moments and reconnected flux; each form is also checked against the FP64
    oracle with the same splitting over 2 steps on the central 16 x 8
    subdomain."""
    import numpy as np

    import oracle
    from oracle.step import OracleState
    from paper_2109_06743_gb300.driver import Simulation
    oracle.build()
    out = {"run": "harris 64x32 x 16^3 subdomain (dx, dv, dt of harris_512x256_v16), FP64, fitted, %d steps" % steps}
    mom = {}
    for ns in (5, 3):
        cfg = make_cfg("harris_512x256_v16", precision=64, sub=(64, 32))
        cfg.nshear = ns
        sim = Simulation(cfg, initial_state(cfg, np.float64), None, initial_yee(cfg), device=device)
        e0, psi0 = sim.total_energy(), sim.reconnected_flux(0.0)
        for _ in range(steps):
            sim.step()
        mom[ns] = [m.cpu().numpy() for m in sim.mom_t]
        out["shears_%d" % ns] = {"energy_drift": (sim.total_energy() - e0) / e0,
                                 "reconnected_flux_change": sim.reconnected_flux(0.0) - psi0}
        sim.close()
        # parity of this splitting with the oracle's
        cs = make_cfg("harris_512x256_v16", precision=64, sub=(16, 8))
        cs.nshear = ns
        f0 = initial_state(cs, np.float64)
        g = Simulation(cs, f0, None, initial_yee(cs), device=device)
        o = OracleState(cs, f0, None, initial_yee(cs))
        for _ in range(2):
            g.step()
            o.step(cs.dt)
        out["shears_%d" % ns]["f_max_rel_diff_vs_oracle_16x8_2_steps"] = max(
            float(np.abs(g.f_host(k) - o.f[k]).max() / o.f[k].max()) for k in range(2))
        g.close()
    # moments of the two runs: largest difference relative to the moment's
    # largest magnitude over the grid
    diffs = []
    for a, b in zip(mom[5], mom[3]):
        sc = np.abs(a).max(axis=0) + 1e-300
        diffs.append(float((np.abs(a - b) / sc).max()))
    out["moments_max_rel_diff_3_vs_5"] = max(diffs)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="harris_512x256_v16", choices=sorted(WORKLOADS) + [LANDAU])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=10, help="steps of the FP64 form timed for comparison")
    ap.add_argument("--no-mlp", action="store_true", help="cold-started fits only (no warm-start network)")
    ap.add_argument("--single-axis", action="store_true",
                    help="the spatial step as two single-axis sweeps (pfc_advect_x) instead of the fused x+y one")
    ap.add_argument("--train-from", default=None, choices=sorted(WORKLOADS),
                    help="workload whose fits train the warm-start network (default: the same velocity grid)")
    ap.add_argument("--harvest-steps", type=int, default=24, help="cold-started steps harvested for training")
    ap.add_argument("--no-all-cores", action="store_true", help="skip the all-cores oracle figure")
    ap.add_argument("--no-extra", action="store_true",
                    help="only the named workload: no nested lines of the other workloads, no network transfer, "
                         "no shear ablation")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == LANDAU:
        return run_landau(args, rank)

    import torch

    from paper_2109_06743_gb300 import abi
    from paper_2109_06743_gb300 import build as B

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
    alu = measured_alu_peaks(device)
    extra = not args.no_extra and args.workload == "harris_512x256_v16"
    # the end-to-end leg times the same K steps as the device figure (each
    # run; at most 50)
    res = measure_2d3v(args.workload, device, alu, args.steps, args.warmup, 0 if args.no_e2e else min(args.steps, 50),
                       max(1, min(args.steps, 5)), args.fp64_steps, not args.no_cpu, not args.no_all_cores,
                       harvest_steps=args.harvest_steps, train_from=args.train_from, no_mlp=args.no_mlp, dist=dist,
                       world=world, gpu_index=local,
                       transfer_from="harris_128x64_v20" if extra and not args.no_mlp else None,
                       transfer_samples=10_000_000, fused_xy=not args.single_axis)
    line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    line.update({k: v for k, v in res.items() if k not in ("value", "steps", "warmup", "ms_per_step")})
    line["config"]["host_cores"] = affinity
    line["alu_peaks"] = alu
    if extra:
        # the other workloads of the metric, a few timed steps each (rank 0's
        # GPU; under torchrun the other ranks time their own replicas alike)
        nested = {}
        nested["asym_1024x512_v12"] = measure_2d3v(
            "asym_1024x512_v12", device, alu, 5, 2, 3, 3, 3 if args.fp64_steps else 0, not args.no_cpu, False,
            dist=dist, world=world, gpu_index=local)
        # the 20^3 Harris run whose fits train the transfer network (no
        # accuracy window: its oracle step would take minutes on one core)
        nested["harris_128x64_v20"] = measure_2d3v(
            "harris_128x64_v20", device, alu, 10, 3, 10, 3, 3 if args.fp64_steps else 0, False, False,
            dist=dist, world=world, gpu_index=local)
        if rank == 0:
            nested[LANDAU] = landau_block(200, 3)
            line["shear_ablation"] = shear_ablation(device)
            line["species_launch_fixed_cost"] = launch_fixed_cost(
                device, res["ms_per_step"], {k: v["ms_per_launch"] for k, v in res["hbm_phases"].items()})
        line["workloads"] = nested
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
