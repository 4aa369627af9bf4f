"""Algorithm 1 of the paper (Sec. 2.2) driven through the C-ABI.

``Simulation`` owns the device buffers (allocated with PyTorch: plumbing only)
and enqueues one time step as a sequence of libvlasov calls on one CUDA
stream, with no host synchronisation inside a step:

2D3V (Lie splitting x, y, v):
  1. maxwell_step(dt/2)            current of the fluid state
  2. Q^t                           moments of f^t (from the previous exchange)
  then species by species:
  3. pfc_advect_xy (x then y in one out-of-place pass; the two buffers of a
     species swap roles), pfc_advect_v(+ moments -> Q^t+1, V targets)
  4. fluid_step_species(dt, Q^t, Q^t+1)  SSP-RK3, Q^t+1/2 = average, with the
     fields frozen (a species' fluid state needs only its own moments)
  5. moment_fit                    Newton fits, exchange, limiter (+ moments of the new f)
  and then
  6. maxwell_step(dt/2)            current of the fitted moments
1D1V (Strang x/2, v, x/2; Poisson instead of FDTD, Sec. 3.1): E from the
density after the first half x sweep.
"""
from __future__ import annotations

import numpy as np

from . import abi
from . import workloads as W


class Simulation:
    def __init__(self, cfg, f_list, fluid_list=None, yee=None, device="cuda", stream=None, fit=True,
                 fused_xy=True, wide_fit=None):
        """wide_fit: which double-float Newton kernel the FP32-mode fits use
        (moment_fit_wide): None lets the library choose it on the device at
        every fit from the targets; True/False forces the kernel with the
        centre-out evaluation (Maxwellians narrow against their velocity box)
        or the common one for every species."""
        import torch

        self.torch = torch
        self.cfg = cfg
        self.dev = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.dev)
        self.fit = fit
        self.fused_xy = fused_xy and cfg.nvdim == 3
        self.dtype = torch.float32 if cfg.precision == 32 else torch.float64
        nvdim, nc = cfg.nvdim, cfg.ncell
        self.nmom = 4 if nvdim == 1 else 20
        self.ncomp = 3 if nvdim == 1 else 10
        with torch.cuda.stream(self.stream):
            self.f = []
            for f in f_list:
                t = torch.as_tensor(np.asarray(f)).reshape(nc, -1).to(device=self.dev, dtype=self.dtype)
                self.f.append(t.contiguous())
            # second buffer per species for the out-of-place x+y sweep
            self.f_spare = [torch.empty_like(t) for t in self.f] if self.fused_xy else None
            self.fluid = torch.zeros((len(cfg.species), nc, self.ncomp), dtype=torch.float64, device=self.dev)
            self.eb = torch.zeros((nc, 6), dtype=torch.float64, device=self.dev)
            if nvdim == 3:
                y = np.zeros((6, cfg.ny + 1, cfg.nx)) if yee is None else np.asarray(yee, dtype=np.float64)
                self.yee = torch.as_tensor(y.reshape(-1)).to(self.dev).contiguous()
            else:
                self.yee = None
            self.desc = abi.make_desc(cfg)
            self.work_bytes = abi.vlasov_work_bytes(self.desc)
            if self.work_bytes == 0:
                raise abi.VlasovError(abi.VL_EINVAL, abi.lib().vl_last_error(None).decode())
            self.work = torch.zeros(self.work_bytes + 256, dtype=torch.uint8, device=self.dev)
            off = (-self.work.data_ptr()) % 256
            self.work_ptr = self.work.data_ptr() + off
            self.mom_t = [torch.zeros((nc, self.nmom), dtype=torch.float64, device=self.dev) for _ in cfg.species]
            self.mom_t1 = [torch.zeros((nc, self.nmom), dtype=torch.float64, device=self.dev) for _ in cfg.species]
            self.mom_tmp = [torch.zeros((nc, self.nmom), dtype=torch.float64, device=self.dev) for _ in cfg.species]
        self.ctx = abi.vlasov_init(self.desc, self.f, self.fluid, self.yee, self.eb, self.work_ptr, self.work_bytes)
        s = self.stream
        for k in range(len(cfg.species)):
            abi.moments(self.ctx, k, self.mom_t[k], s)
        with torch.cuda.stream(s):
            if fluid_list is None:
                # the fluid starts from the moments of f, so both solvers agree
                for k in range(len(cfg.species)):
                    self.fluid[k].copy_(self.mom_t[k][:, :self.ncomp])
            else:
                for k, u in enumerate(fluid_list):
                    self.fluid[k].copy_(torch.as_tensor(np.asarray(u).reshape(nc, self.ncomp)))
        if nvdim == 3:
            abi.maxwell_step(self.ctx, 0.0, None, s)  # cell-centred fields of the initial Yee fields
        else:
            abi.maxwell_step(self.ctx, 0.0, self.mom_t, s)
        self.wide_fit = wide_fit
        if nvdim == 3 and fit and wide_fit is not None:
            for k in range(len(cfg.species)):
                abi.moment_fit_wide(self.ctx, k, wide_fit)
        self.time = 0.0
        self.nstep = 0

    def close(self):
        if self.ctx is not None:
            abi.vlasov_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- Algorithm 1 -----------------------------------------------------------
    def step(self, dt=None, use_mlp=False, mark=None, first_use=None, last_use=None):
        """One time step. ``mark(label)``, if given, is called before each
        phase (the benchmark records a CUDA event there); ``first_use(k)`` and
        ``last_use(k)``, if given, are called right before the first and
        right after the last kernel of the step that touches f of species k
        (step_through_host hangs its copies there). None of them changes the
        work."""
        cfg, ctx, s = self.cfg, self.ctx, self.stream
        dt = cfg.dt if dt is None else dt
        ns = len(cfg.species)
        mark = mark or (lambda label: None)
        first_use = first_use or (lambda k: None)
        last_use = last_use or (lambda k: None)
        if cfg.nvdim == 1:
            abi.maxwell_step(ctx, 0.5 * dt, self.mom_t, s)
            for k in range(ns):
                first_use(k)
                abi.pfc_advect_x(ctx, k, 0, 0.5 * dt, s)
                abi.moments(ctx, k, self.mom_tmp[k], s)
            abi.maxwell_step(ctx, 0.5 * dt, self.mom_tmp, s)
            for k in range(ns):
                abi.pfc_advect_v(ctx, k, dt, None, s)
                abi.pfc_advect_x(ctx, k, 0, 0.5 * dt, s)
                abi.moments(ctx, k, self.mom_t1[k], s)
                if not self.fit:
                    last_use(k)
        else:
            mark("maxwell")
            abi.maxwell_step(ctx, 0.5 * dt, None if self.fit else self.mom_t, s)
            for k in range(ns):
                first_use(k)
                if self.fused_xy:
                    mark("xy_sweep")
                    abi.pfc_advect_xy(ctx, k, dt, self.f_spare[k], s)
                    self.f[k], self.f_spare[k] = self.f_spare[k], self.f[k]
                else:
                    mark("x_sweep")
                    abi.pfc_advect_x(ctx, k, 0, dt, s)
                    mark("y_sweep")
                    abi.pfc_advect_x(ctx, k, 1, dt, s)
                mark("v_pass")
                abi.pfc_advect_v(ctx, k, dt, self.mom_t1[k], s)
                if self.fit:
                    # the species' own fluid step, fit and exchange before the
                    # next species' sweeps (each fluid state needs only its own
                    # moments and the frozen fields), so that its f is final,
                    # and can start its way to the host, as early as possible
                    mark("fluid")
                    abi.fluid_step_species(ctx, k, dt, self.mom_t[k], self.mom_t1[k], s)
                    mark("fit_solve")
                    abi.moment_fit_solve(ctx, k, self.mom_t1[k], use_mlp, None, None, s)
                    mark("fit_exchange")
                    abi.moment_fit_exchange(ctx, k, self.mom_t1[k], self.mom_t[k], s)
                last_use(k)
        if self.fit and cfg.nvdim == 1:
            mark("fluid")
            abi.fluid_step(ctx, dt, self.mom_t, self.mom_t1, s)
            for k in range(ns):
                mark("fit_solve")
                abi.moment_fit_solve(ctx, k, self.mom_t1[k], use_mlp, None, None, s)
                mark("fit_exchange")
                abi.moment_fit_exchange(ctx, k, self.mom_t1[k], self.mom_t[k], s)
                last_use(k)
        elif not self.fit:
            self.mom_t, self.mom_t1 = self.mom_t1, self.mom_t
        mark("maxwell")
        if cfg.nvdim == 1:
            abi.maxwell_step(ctx, 0.5 * dt, self.mom_t, s)
        else:
            abi.maxwell_step(ctx, 0.5 * dt, None if self.fit else self.mom_t, s)
        mark(None)
        self.time += dt
        self.nstep += 1

    def graph(self, steps, use_mlp=False):
        """A CUDA graph of `steps` time steps on the solver's stream, to be
        replayed with .replay() (for launch-bound workloads such as the 1D1V
        runs, whose kernels take a few microseconds each). The stream must be
        a created stream, not the legacy default one; with the fused x+y
        sweep `steps` must be even, so that each species' two buffers end
        where they started. A step must have run before (first-launch
        set-up); replays do not advance self.time, and a replay runs on the
        current stream (replay inside `with torch.cuda.stream(sim.stream)`
        to keep it ordered with the solver's other work)."""
        torch = self.torch
        if self.stream == torch.cuda.default_stream(self.dev):
            raise ValueError("capture needs a created stream (Simulation(..., stream=torch.cuda.Stream()))")
        if self.fused_xy and steps % 2:
            raise ValueError("with the fused x+y sweep the captured step count must be even")
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            for _ in range(steps):
                self.step(use_mlp=use_mlp)
        self.time -= steps * self.cfg.dt
        return g

    # pieces per species of the host copies: the copy in of piece c of the
    # next step follows the copy out of piece c of this one, so the two
    # directions pipeline
    HOST_CHUNKS = 8

    def step_through_host(self, host, use_mlp=False):
        """One step whose f comes from, and goes back to, pinned host buffers
        host[k] (the end-to-end form). The copy of species k into the device
        runs on its own stream and is awaited right before the species' first
        kernel; its copy back starts as soon as the species' last kernel has
        finished, on another stream; and the next step's copy in waits for it.
        So one species' transfers overlap the other species' kernels, and the
        two directions overlap each other."""
        torch = self.torch
        ns = len(self.cfg.species)
        self.host_streams_after(None)
        nch = self.HOST_CHUNKS
        h2d_done = [None] * ns
        for k in range(ns):
            dev_parts, host_parts = self.f[k].chunk(nch), host[k].chunk(nch)
            with torch.cuda.stream(self._h2d):
                for c in range(len(dev_parts)):
                    # chunk c of the previous step's copy back must have left
                    if self._d2h_done[k] is not None:
                        self._h2d.wait_event(self._d2h_done[k][c])
                    dev_parts[c].copy_(host_parts[c], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self._h2d)
                h2d_done[k] = ev

        def first_use(k):
            self.stream.wait_event(h2d_done[k])

        def last_use(k):
            ev = torch.cuda.Event()
            ev.record(self.stream)
            dev_parts, host_parts = self.f[k].chunk(nch), host[k].chunk(nch)
            done = []
            with torch.cuda.stream(self._d2h):
                self._d2h.wait_event(ev)
                for c in range(len(dev_parts)):
                    host_parts[c].copy_(dev_parts[c], non_blocking=True)
                    e = torch.cuda.Event()
                    e.record(self._d2h)
                    done.append(e)
            self._d2h_done[k] = done

        self.step(use_mlp=use_mlp, first_use=first_use, last_use=last_use)

    def host_streams_after(self, event):
        """Create the copy streams of step_through_host if needed and, given
        an event, make them wait for it (a timer's start)."""
        torch = self.torch
        if getattr(self, "_h2d", None) is None:
            self._h2d = torch.cuda.Stream(self.dev)
            self._d2h = torch.cuda.Stream(self.dev)
            self._d2h_done = [None] * len(self.cfg.species)
        if event is not None:
            self._h2d.wait_event(event)
            self._d2h.wait_event(event)

    def wait_host(self):
        """Make the solver's stream wait for the last copies back to the host."""
        for evs in getattr(self, "_d2h_done", None) or []:
            for ev in evs or []:
                self.stream.wait_event(ev)

    # -- checkpoint and resume ------------------------------------------------------
    def save(self, path):
        """Write everything that determines the later steps to ``path`` (an
        .npz file): f of every species, the fluid state, the moments of f at t
        (from the last exchange: the next step's Q^t), the Yee and the
        cell-centred fields, the time and step count, the warm-start network's
        parameters (when the context has them) and the configuration. A
        Simulation made by ``resume`` from it continues bit for bit as this
        one would. Synchronises the stream."""
        cfg = self.cfg
        self.stream.synchronize()
        arrays = {"config": np.array(W.config_to_json(cfg)), "time": np.array(self.time),
                  "nstep": np.array(self.nstep), "fit": np.array(self.fit),
                  "fluid": self.fluid.cpu().numpy(), "eb": self.eb.cpu().numpy()}
        try:
            arrays["mlp"] = abi.mlp_get_weights(self.ctx)
        except abi.VlasovError:
            pass  # the context has no network
        for k in range(len(cfg.species)):
            arrays["f%d" % k] = self.f[k].cpu().numpy()
            arrays["mom_t%d" % k] = self.mom_t[k].cpu().numpy()
        if self.yee is not None:
            arrays["yee"] = self.yee.cpu().numpy()
        np.savez(path, **arrays)

    @classmethod
    def resume(cls, path, device="cuda", stream=None, fused_xy=True, wide_fit=None):
        """A Simulation in the state ``save`` wrote to ``path``."""
        import torch

        z = np.load(path)
        cfg = W.config_from_json(str(z["config"]))
        ns = len(cfg.species)
        sim = cls(cfg, [z["f%d" % k] for k in range(ns)], list(z["fluid"]), z["yee"] if "yee" in z else None,
                  device=device, stream=stream, fit=bool(z["fit"]), fused_xy=fused_xy, wide_fit=wide_fit)
        with torch.cuda.stream(sim.stream):
            for k in range(ns):
                sim.mom_t[k].copy_(torch.as_tensor(z["mom_t%d" % k]))
            sim.eb.copy_(torch.as_tensor(z["eb"]))
            if "yee" in z:
                # the constructor's zero-length field step may turn -0.0 into +0.0
                sim.yee.copy_(torch.as_tensor(z["yee"]))
        if "mlp" in z:
            abi.mlp_set_weights(sim.ctx, z["mlp"])
        sim.time = float(z["time"])
        sim.nstep = int(z["nstep"])
        return sim

    # -- per-step diagnostics ------------------------------------------------------
    def diagnostics(self):
        """Step, time, mass per species (m times the integral of n), energy
        partition and total, the reconnected flux (2D3V) and the fit counters
        accumulated since the last reset (Newton iterations, fallbacks,
        clipped cells, invalid targets). Synchronises the stream."""
        cfg = self.cfg
        kin, ee, eb = self.energies()
        area = cfg.dx * (cfg.dy if cfg.nvdim == 3 else 1.0)
        st = self.stats()
        d = {"step": self.nstep, "time": self.time,
             "mass": [float(m[:, 0].sum().item()) * area * sp.m for sp, m in zip(cfg.species, self.mom_t)],
             "kinetic_thermal": [float(x) for x in kin], "electric": float(ee), "magnetic": float(eb),
             "total_energy": float(sum(kin) + ee + eb),
             "newton_iterations": st[0], "newton_fallbacks": st[1], "clipped_cells": st[2], "invalid_fits": st[3]}
        if cfg.nvdim == 3:
            # on the sheet's X line (the B_x null of an asymmetric sheet)
            d["reconnected_flux"] = float(self.reconnected_flux(W.x_line(cfg) if hasattr(cfg, "kind") else 0.0))
        return d

    def run(self, steps, use_mlp=False, log=None, every=1):
        """Advance ``steps`` steps. With ``log`` (a path, opened for appending,
        or a text file), write one JSON line of ``diagnostics()`` every
        ``every`` steps and after the last one, with the fit counters of the
        steps since the previous line and the mean step time over them (CUDA
        events on the solver's stream, diagnostics excluded)."""
        import json

        torch = self.torch
        fh = open(log, "a") if isinstance(log, (str, bytes)) or hasattr(log, "__fspath__") else log
        try:
            if fh is not None:
                abi.vl_reset_stats(self.ctx, self.stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            since = 0
            for i in range(steps):
                self.step(use_mlp=use_mlp)
                since += 1
                if fh is not None and (since == every or i == steps - 1):
                    e1.record(self.stream)
                    e1.synchronize()
                    d = self.diagnostics()
                    d["ms_per_step"] = e0.elapsed_time(e1) / since
                    fh.write(json.dumps(d) + "\n")
                    fh.flush()
                    abi.vl_reset_stats(self.ctx, self.stream)
                    since = 0
                    e0.record(self.stream)
        finally:
            if fh is not None and fh is not log:
                fh.close()

    # -- host-side views (diagnostics and tests) --------------------------------
    def f_host(self, k):
        return self.f[k].double().cpu().numpy()

    def stats(self):
        return abi.vl_read_stats(self.ctx, self.stream)

    def energies(self):
        """(kinetic+thermal per species, electric, magnetic) from the moments
        of f at t and the fields, summed on the host (diagnostic only)."""
        cfg = self.cfg
        self.stream.synchronize()
        area = cfg.dx * (cfg.dy if cfg.nvdim == 3 else 1.0)
        kin = []
        for sp, m in zip(cfg.species, self.mom_t):
            m = m.cpu().numpy()
            v2 = m[:, 2] if cfg.nvdim == 1 else m[:, 4] + m[:, 7] + m[:, 9]
            kin.append(0.5 * sp.m * v2.sum() * area)
        if cfg.nvdim == 1:
            e = self.eb[:, 0].cpu().numpy()
            return kin, 0.5 * (e ** 2).sum() * area, 0.0
        y = self.yee.cpu().numpy().reshape(6, cfg.ny + 1, cfg.nx)
        rows = slice(0, cfg.ny + 1) if cfg.bc_y == 1 else slice(0, cfg.ny)
        eps0 = 1.0 / cfg.c ** 2
        ee = 0.5 * eps0 * ((y[0, rows] ** 2).sum() + (y[1, :cfg.ny] ** 2).sum() + (y[2, rows] ** 2).sum()) * area
        eb = 0.5 * ((y[3, :cfg.ny] ** 2).sum() + (y[4, rows] ** 2).sum() + (y[5, :cfg.ny] ** 2).sum()) * area
        return kin, ee, eb

    def total_energy(self):
        kin, ee, eb = self.energies()
        return sum(kin) + ee + eb

    def reconnected_flux(self, y_line=0.0):
        """Reconnected flux of the GEM set-up (Sec. 3.3): with B_y = -dA_z/dx
        on the sheet's midline (the integer Yee row nearest y_line: y = 0 for
        a symmetric sheet, the B_x null of an asymmetric one), half the
        integral of |B_y| over x, i.e. max A_z - min A_z along the midline for
        one X and one O point (diagnostic only)."""
        cfg = self.cfg
        self.stream.synchronize()
        y = self.yee.cpu().numpy().reshape(6, cfg.ny + 1, cfg.nx)
        jm = int(round((y_line - cfg.y0) / cfg.dy))
        return 0.5 * np.abs(y[4, jm]).sum() * cfg.dx


class ClosureFluid:
    """The stand-alone ten-moment fluid model with the gradient heat-flux
    closure (Sec. 2.3) through the C-ABI, on a fluid-only context (no f):
    per step maxwell_step(dt/2) with the current of the fluid state,
    fluid_step_closure(dt), maxwell_step(dt/2). 2D3V."""

    def __init__(self, cfg, fluid_list, yee, device="cuda", stream=None):
        import torch

        self.torch = torch
        self.cfg = cfg
        self.dev = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.dev)
        nc = cfg.ncell
        with torch.cuda.stream(self.stream):
            self.fluid = torch.as_tensor(np.stack([np.asarray(u, dtype=np.float64).reshape(nc, 10)
                                                   for u in fluid_list])).to(self.dev).contiguous()
            self.eb = torch.zeros((nc, 6), dtype=torch.float64, device=self.dev)
            self.yee = torch.as_tensor(np.asarray(yee, dtype=np.float64).reshape(-1)).to(self.dev).contiguous()
            self.desc = abi.make_desc(cfg)
            self.work_bytes = abi.vlasov_work_bytes(self.desc)
            if self.work_bytes == 0:
                raise abi.VlasovError(abi.VL_EINVAL, abi.lib().vl_last_error(None).decode())
            self.work = torch.zeros(self.work_bytes + 256, dtype=torch.uint8, device=self.dev)
            self.work_ptr = self.work.data_ptr() + (-self.work.data_ptr()) % 256
        self.ctx = abi.vlasov_init(self.desc, None, self.fluid, self.yee, self.eb, self.work_ptr, self.work_bytes)
        abi.maxwell_step(self.ctx, 0.0, None, self.stream)  # cell-centred fields
        self.time = 0.0

    def step(self, dt=None):
        dt = self.cfg.dt if dt is None else dt
        abi.maxwell_step(self.ctx, 0.5 * dt, None, self.stream)
        abi.fluid_step_closure(self.ctx, dt, self.stream)
        abi.maxwell_step(self.ctx, 0.5 * dt, None, self.stream)
        self.time += dt

    def energies(self):
        """(kinetic+thermal per species = (m/2) sum tr(E2) dA, electric, magnetic)"""
        cfg = self.cfg
        self.stream.synchronize()
        area = cfg.dx * cfg.dy
        U = self.fluid.cpu().numpy()
        kin = [0.5 * sp.m * (U[k, :, 4] + U[k, :, 7] + U[k, :, 9]).sum() * area for k, sp in enumerate(cfg.species)]
        y = self.yee.cpu().numpy().reshape(6, cfg.ny + 1, cfg.nx)
        rows = slice(0, cfg.ny + 1) if cfg.bc_y == 1 else slice(0, cfg.ny)
        eps0 = 1.0 / cfg.c ** 2
        ee = 0.5 * eps0 * ((y[0, rows] ** 2).sum() + (y[1, :cfg.ny] ** 2).sum() + (y[2, rows] ** 2).sum()) * area
        eb = 0.5 * ((y[3, :cfg.ny] ** 2).sum() + (y[4, rows] ** 2).sum() + (y[5, :cfg.ny] ** 2).sum()) * area
        return kin, ee, eb

    def total_energy(self):
        kin, ee, eb = self.energies()
        return sum(kin) + ee + eb

    def close(self):
        if self.ctx is not None:
            abi.vlasov_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
