"""Oracle time step: Algorithm 1 of the paper in plain FP64 (test infrastructure only).

Algorithm 1 (Sec. 2.2), as implemented here:

  1. half step of the field solver (FDTD with the current of the fluid state;
     1D1V: Poisson solve),
  2. third moment Q^t from f^t,
  3. Vlasov step f^t -> f^{t+1} (spatial PFC sweeps, velocity PFC shears),
  4. Q^{t+1} from f^{t+1},
  5. Q^{t+1/2} = (Q^t + Q^{t+1}) / 2,
  6. SSP-RK3 fluid step with Q at t, t+dt, t+dt/2 and E, B at t+dt/2,
  7. moment fitting (Newton fits of the V and F Maxwellians, exchange, limit),
  8. second field half step with the current of the fitted moments.

Readings where the paper is silent: Lie splitting x, y, v
for 2D3V and Strang splitting x/2, v, x/2 for 1D1V; the fluid state is replaced
by its rescaled moments after fitting; E in 1D1V from the density of f after
the first half x-sweep.
"""
from __future__ import annotations

import numpy as np

from . import (Grid, advect_space, advect_velocity, closure_chi_k0, fields_to_centres, fluid_step,
               fluid_step_closure, make_grid, make_species, maxwell, moment_fit, moments, poisson_1d)


def grid_of(cfg) -> Grid:
    return make_grid(cfg.nvdim, cfg.nx, cfg.ny, cfg.x0, cfg.dx, cfg.y0, cfg.dy, cfg.bc_y)


def species_of(sp):
    return make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)


def third_moments(mom, nvdim):
    return np.ascontiguousarray(mom[:, 3:4] if nvdim == 1 else mom[:, 10:20])


class OracleState:
    """State of the oracle solver: f per species (float64), fluid U per
    species, Yee fields (2D3V) or cell-centred E (1D1V)."""

    def __init__(self, cfg, f_list, fluid_list=None, yee=None):
        self.cfg = cfg
        self.g = grid_of(cfg)
        self.sps = [species_of(s) for s in cfg.species]
        self.f = [np.ascontiguousarray(f, dtype=np.float64).reshape(cfg.ncell, -1).copy() for f in f_list]
        ncomp = 3 if cfg.nvdim == 1 else 10
        if fluid_list is None:
            # the fluid starts from the moments of f, so both solvers agree
            fluid_list = [moments(f, self.g, sp)[:, :ncomp].copy() for f, sp in zip(self.f, self.sps)]
        self.U = [np.ascontiguousarray(u, dtype=np.float64).reshape(cfg.ncell, ncomp).copy() for u in fluid_list]
        self.yee = None if yee is None else np.ascontiguousarray(yee, dtype=np.float64).reshape(-1).copy()
        self.EB = np.zeros((cfg.ncell, 6))
        self.stats = np.zeros(3, dtype=np.int64)
        self.time = 0.0
        if cfg.nvdim == 3:
            self.EB = fields_to_centres(self.yee, self.g)
        else:
            self._poisson_from_f()

    # -- fields -----------------------------------------------------------
    def current(self):
        J = np.zeros((self.cfg.ncell, 3))
        for sp, U in zip(self.cfg.species, self.U):
            J += sp.q * U[:, 1:4]
        return J

    def _poisson_from_f(self):
        cfg = self.cfg
        rho = np.full(cfg.nx, cfg.ion_background)
        for sp, s, f in zip(cfg.species, self.sps, self.f):
            rho += sp.q * moments(f, self.g, s)[:, 0]
        self.EB[:, 0] = poisson_1d(rho, cfg.dx)

    def field_half(self, h):
        if self.cfg.nvdim == 1:
            self._poisson_from_f()
            return
        maxwell(self.yee, self.g, self.current(), h, self.cfg.c)
        self.EB = fields_to_centres(self.yee, self.g)

    # -- one step of Algorithm 1 -------------------------------------------
    def step(self, dt, fit=True):
        cfg = self.cfg
        d = cfg.nvdim
        self.field_half(0.5 * dt)
        Q0 = [third_moments(moments(f, self.g, s), d) for f, s in zip(self.f, self.sps)]
        for f, s in zip(self.f, self.sps):
            if d == 1:
                advect_space(f, self.g, s, 0, 0.5 * dt)
            else:
                advect_space(f, self.g, s, 0, dt)
                advect_space(f, self.g, s, 1, dt)
        if d == 1:
            self._poisson_from_f()
        for f, s in zip(self.f, self.sps):
            advect_velocity(f, self.g, s, self.EB, dt, cfg.nshear)
            if d == 1:
                advect_space(f, self.g, s, 0, 0.5 * dt)
        Q1 = [third_moments(moments(f, self.g, s), d) for f, s in zip(self.f, self.sps)]
        if fit:
            EBfl = self.EB.copy()
            for k, (U, s) in enumerate(zip(self.U, self.sps)):
                Qh = 0.5 * (Q0[k] + Q1[k])
                fluid_step(U, self.g, s, Q0[k], Qh, Q1[k], EBfl, dt)
            for f, U, s in zip(self.f, self.U, self.sps):
                st = moment_fit(f, self.g, s, U, cfg.fit_tol, cfg.fit_max_iter)
                self.stats += np.array(st, dtype=np.int64)
        else:
            ncomp = 3 if d == 1 else 10
            for k, (f, s) in enumerate(zip(self.f, self.sps)):
                self.U[k] = moments(f, self.g, s)[:, :ncomp].copy()
        self.field_half(0.5 * dt)
        self.time += dt

    # -- diagnostics ------------------------------------------------------
    def energies(self):
        """(kinetic+thermal per species, electric, magnetic), each summed over
        space; kinetic+thermal = (m/2) int v^2 f (Sec. 3.2 energy partition)."""
        cfg = self.cfg
        area = cfg.dx * (cfg.dy if cfg.nvdim == 3 else 1.0)
        kin = []
        for sp, s, f in zip(cfg.species, self.sps, self.f):
            mom = moments(f, self.g, s)
            v2 = mom[:, 2] if cfg.nvdim == 1 else mom[:, 4] + mom[:, 7] + mom[:, 9]
            kin.append(0.5 * sp.m * v2.sum() * area)
        if cfg.nvdim == 1:
            ee = 0.5 * (self.EB[:, 0] ** 2).sum() * area
            return kin, ee, 0.0
        yee = self.yee.reshape(6, cfg.ny + 1, cfg.nx)
        eps0 = 1.0 / cfg.c ** 2
        rows_int = slice(0, cfg.ny + 1) if cfg.bc_y == 1 else slice(0, cfg.ny)
        ee = 0.5 * eps0 * ((yee[0, rows_int] ** 2).sum() + (yee[1, :cfg.ny] ** 2).sum()
                           + (yee[2, rows_int] ** 2).sum()) * area
        eb = 0.5 * ((yee[3, :cfg.ny] ** 2).sum() + (yee[4, rows_int] ** 2).sum()
                    + (yee[5, :cfg.ny] ** 2).sum()) * area
        return kin, ee, eb

    def total_energy(self):
        kin, ee, eb = self.energies()
        return sum(kin) + ee + eb

    def reconnected_flux(self, y_line=0.0):
        """psi = (1/2) sum_x |B_y(x, y_line)| dx on the integer Yee row nearest
        the midline y_line (GEM diagnostic, Sec. 3.3)."""
        cfg = self.cfg
        By = self.yee.reshape(6, cfg.ny + 1, cfg.nx)[4]
        row = int(round((y_line - cfg.y0) / cfg.dy))
        return 0.5 * float(np.sum(np.abs(By[row]))) * cfg.dx

    def mass(self):
        cfg = self.cfg
        return [moments(f, self.g, s)[:, 0].sum() for f, s in zip(self.f, self.sps)]


class OracleClosureFluid:
    """The stand-alone ten-moment fluid with the gradient heat-flux closure
    (Sec. 2.3) coupled to the FDTD fields: per step a field half step with
    the current of the fluid state, one SSP-RK3 fluid step with E and B
    frozen, and a second field half step (the order of Algorithm 1 without
    the kinetic part). 2D3V."""

    def __init__(self, cfg, fluid_list, yee, chi_scale=1.0):
        self.cfg = cfg
        self.g = grid_of(cfg)
        self.sps = [species_of(s) for s in cfg.species]
        self.U = [np.ascontiguousarray(u, dtype=np.float64).reshape(cfg.ncell, 10).copy() for u in fluid_list]
        self.yee = np.ascontiguousarray(yee, dtype=np.float64).reshape(-1).copy()
        self.EB = fields_to_centres(self.yee, self.g)
        self.chi_k0 = [chi_scale * closure_chi_k0(sp.q, sp.m) for sp in cfg.species]
        self.time = 0.0

    def current(self):
        J = np.zeros((self.cfg.ncell, 3))
        for sp, U in zip(self.cfg.species, self.U):
            J += sp.q * U[:, 1:4]
        return J

    def field_half(self, h):
        maxwell(self.yee, self.g, self.current(), h, self.cfg.c)
        self.EB = fields_to_centres(self.yee, self.g)

    def step(self, dt):
        self.field_half(0.5 * dt)
        EB = self.EB.copy()
        for U, s, ck in zip(self.U, self.sps, self.chi_k0):
            fluid_step_closure(U, self.g, s, EB, dt, ck)
        self.field_half(0.5 * dt)
        self.time += dt

    def energies(self):
        """(kinetic+thermal per species = (m/2) sum tr(E2) dA, electric, magnetic)"""
        cfg = self.cfg
        area = cfg.dx * cfg.dy
        kin = [0.5 * sp.m * (U[:, 4] + U[:, 7] + U[:, 9]).sum() * area for sp, U in zip(cfg.species, self.U)]
        yee = self.yee.reshape(6, cfg.ny + 1, cfg.nx)
        eps0 = 1.0 / cfg.c ** 2
        rows_int = slice(0, cfg.ny + 1) if cfg.bc_y == 1 else slice(0, cfg.ny)
        ee = 0.5 * eps0 * ((yee[0, rows_int] ** 2).sum() + (yee[1, :cfg.ny] ** 2).sum()
                           + (yee[2, rows_int] ** 2).sum()) * area
        eb = 0.5 * ((yee[3, :cfg.ny] ** 2).sum() + (yee[4, rows_int] ** 2).sum()
                    + (yee[5, :cfg.ny] ** 2).sum()) * area
        return kin, ee, eb

    def total_energy(self):
        kin, ee, eb = self.energies()
        return sum(kin) + ee + eb
