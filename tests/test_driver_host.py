"""Host logic of the driver, on the CPU: the choice of the wide fit kernel
from the moments of f (Simulation.wide_species), which picks it for the
asymmetric sheet (velocity boxes sized for the hot side: the cold side's
Maxwellians fall by ~112 e-folds into the box corners) and not for the
Harris sheet (boxes of +-5 thermal speeds: ~40 e-folds)."""
import types

import numpy as np
import pytest

from paper_2109_06743_gb300 import workloads as W


def fake_sim(orc, cfg, f_list):
    import torch
    g = orc.make_grid(3, cfg.nx, cfg.ny, cfg.x0, cfg.dx, cfg.y0, cfg.dy, cfg.bc_y)
    mom = []
    for sp, f in zip(cfg.species, f_list):
        s = orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)
        mom.append(torch.as_tensor(orc.moments(np.ascontiguousarray(f.reshape(cfg.ncell, -1)), g, s)))
    from paper_2109_06743_gb300.driver import Simulation
    return types.SimpleNamespace(cfg=cfg, mom_t=mom, torch=torch, stream=None, WIDE_SPREAD=Simulation.WIDE_SPREAD)


@pytest.mark.parametrize("kind,want", [("asym", True), ("harris", False)])
def test_wide_fit_kernel_choice(orc, kind, want):
    from paper_2109_06743_gb300.driver import Simulation
    if kind == "asym":
        cfg = W.asym_sheet(nx=4, ny=16, nv=12, lx=0.8, ly=6.4)
        f = W.asym_state(cfg)
    else:
        cfg = W.harris(nx=8, ny=16, nv=12)  # the full 25.6 x 12.8 box: a weak X-line current
        f = W.harris_state(cfg)
    assert Simulation.wide_species(fake_sim(orc, cfg, f)) == [want, want]


def test_empty_cells_do_not_select_the_wide_kernel(orc):
    """A cell with (numerically) no particles has meaningless moments (here
    a Harris block scaled to 1e-20 of the others): it does not select the
    wide kernel for its species."""
    from paper_2109_06743_gb300.driver import Simulation
    cfg = W.harris(nx=8, ny=16, nv=12)
    f = W.harris_state(cfg)
    f[1][3, 2] *= 1e-20
    f[1][3, 2, 0, 0, 0] = 1e-18  # and lopsided: its "spread" is huge
    sim = fake_sim(orc, cfg, f)
    assert Simulation.wide_species(sim) == [False, False]
