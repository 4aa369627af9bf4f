"""Physics of the GPU path beyond linear Landau damping (Sec. 3.1), and the
standard-PFC ablation (moment fitting off).

* Two-stream instability (64 x 64, v in [-5, 5], [0, 4 pi)): the field at
  k = 0.5 grows at the rate of the dispersion root (within 6%, fitted over
  the exponential phase, 0.01 < |E_k| < 0.1), mass is conserved to 1e-12,
  and the fitted and standard PFC solvers give the same f at t = 30 (L1
  difference below 2%; measured 0.5%), as the paper reports.
* Non-linear Landau damping (32 x 64, v in [-6, 6], alpha = 0.5): mass to
  1e-12, the fitted solver conserves total energy at least five times better
  than standard PFC (measured 0.08% vs 1.4% at t = 30), and the first three
  peaks of the damped field energy agree between the two within 10%.
* Coarse 2D3V wave (12^3 velocity cells): standard PFC heats by more than 1%
  in ten steps while moment fitting keeps the energy to 1e-6 (the paper's
  coarse-grid claim, Sec. 3.2-3.3), on the GPU as in the oracle.
"""
import numpy as np
import pytest

from paper_2109_06743_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2109_06743_gb300 import build
    build.build()
    return torch


def run_1d(cfg, f0, fit, steps):
    from paper_2109_06743_gb300.driver import Simulation
    sim = Simulation(cfg, f0, fit=fit)
    x = cfg.x0 + (np.arange(cfg.nx) + 0.5) * cfg.dx
    E0, m0 = sim.total_energy(), f0[0].sum()
    ts, amps, ee = [], [], []
    for _ in range(steps):
        sim.step()
        e = sim.eb[:, 0].cpu().numpy()
        ts.append(sim.time)
        amps.append(2 * abs(np.sum(e * np.exp(-1j * cfg.k * x))) / cfg.nx)
        ee.append(0.5 * (e ** 2).sum() * cfg.dx)
    f = sim.f_host(0)
    out = {"t": np.array(ts), "amp": np.array(amps), "ee": np.array(ee), "f": f,
           "dE": (sim.total_energy() - E0) / E0, "dm": (f.sum() - m0) / m0}
    sim.close()
    return out


def test_two_stream_growth_rate_and_agreement_with_standard_pfc(gpu):
    from test_oracle_physics import two_stream_root
    cfg = W.two_stream()
    f0 = W.two_stream_state(cfg)
    fit = run_1d(cfg, f0, True, 600)
    std = run_1d(cfg, f0, False, 600)
    _, gamma, _ = two_stream_root(cfg.k)
    # exponential phase: after the initial transient (minimum of |E_k| before
    # t = 8), from |E_k| = 0.01 to 0.1
    a = fit["amp"]
    low = int(np.argmin(a[: int(8 / cfg.dt)]))
    first = low + int(np.argmax(a[low:] > 0.01))
    last = first + int(np.argmax(a[first:] > 0.1))
    rate = np.polyfit(fit["t"][first:last], np.log(a[first:last]), 1)[0]
    assert last - first > 20 and abs(rate - gamma) / gamma < 0.06, (rate, gamma)
    assert abs(fit["dm"]) < 1e-12 and abs(std["dm"]) < 1e-12
    l1 = np.abs(fit["f"] - std["f"]).sum() / np.abs(std["f"]).sum()
    assert l1 < 0.02, l1


def test_nonlinear_landau_fitting_conserves_energy_better(gpu):
    cfg = W.landau(nx=32, nv=64, vmax=6.0, alpha=0.5, steps=600)
    f0 = W.landau_state(cfg)
    fit = run_1d(cfg, f0, True, 600)
    std = run_1d(cfg, f0, False, 600)
    assert abs(fit["dm"]) < 1e-12 and abs(std["dm"]) < 1e-12
    assert abs(fit["dE"]) < 5e-3 and 5 * abs(fit["dE"]) < abs(std["dE"]), (fit["dE"], std["dE"])

    def peaks(r):
        ee = r["ee"][: int(15 / cfg.dt)]
        return np.array([ee[i] for i in range(1, len(ee) - 1) if ee[i] > ee[i - 1] and ee[i] >= ee[i + 1]][:4])

    # the first three peaks of the field energy agree (measured within 6%);
    # by the fourth (1% of the first) the two solvers' dissipation differs
    pf, ps = peaks(fit), peaks(std)
    assert len(pf) == 4 and len(ps) == 4
    assert np.all(np.abs(pf[:3] - ps[:3]) <= 0.1 * ps[:3]), (pf, ps)


def test_standard_pfc_heats_coarse_grid_and_fitting_does_not(gpu):
    from paper_2109_06743_gb300.driver import Simulation
    cfg = W.wave2d(steps=10, precision=64)
    drift = {}
    for fit in (True, False):
        sim = Simulation(cfg, W.wave2d_state(cfg), None, W.wave2d_yee(cfg), fit=fit)
        E0 = sim.total_energy()
        m0 = [sim.f_host(k).sum() for k in range(2)]
        for _ in range(cfg.steps):
            sim.step()
        drift[fit] = (sim.total_energy() - E0) / E0
        for k in range(2):
            assert abs(sim.f_host(k).sum() - m0[k]) <= 1e-12 * m0[k]
        sim.close()
    assert abs(drift[True]) < 1e-6, drift
    assert drift[False] > 1e-2, drift


def test_harris_ablation_energy_error_grows_on_coarser_velocity_grids(gpu):
    """Standard PFC against moment fitting on the GEM/Harris set-up (Sec. 3.3,
    where the paper reports the energy error of standard PFC growing from
    25% at 32^3 to 75% at 18^3 while the fitted solver conserves energy):
    64 x 32 cells on 3.2 x 1.6 d_i (ten cells across the sheet half-width,
    the benchmark's resolution), 20^3 and 12^3 velocity cells, FP64, 150
    steps. The fitted runs keep the total energy to 1e-4 (measured 6e-5:
    the fluid and the Vlasov densities differ by the truncation error of the
    two schemes, and the rescaling by n_V/n_F of Algorithm 1 moves that
    difference into the energy); standard PFC's error is at least ten times
    larger and grows as the velocity grid coarsens."""
    from paper_2109_06743_gb300.driver import Simulation
    drift = {}
    for nv in (20, 12):
        cfg = W.harris(nx=64, ny=32, nv=nv, lx=3.2, ly=1.6, precision=64)
        for fit in (True, False):
            sim = Simulation(cfg, W.harris_state(cfg), None, W.harris_yee(cfg), fit=fit)
            E0 = sim.total_energy()
            for _ in range(150):
                sim.step()
            drift[nv, fit] = (sim.total_energy() - E0) / E0
            sim.close()
    assert abs(drift[20, True]) < 1e-4 and abs(drift[12, True]) < 1e-4, drift
    assert abs(drift[20, False]) > 10 * abs(drift[20, True]), drift
    assert abs(drift[12, False]) > abs(drift[20, False]), drift


def test_asymmetric_sheet_downscaled_reconnection_and_energy_partition(gpu, orc):
    """The asymmetric (magnetopause-like) sheet downscaled to 32 x 16 cells
    over 3.2 x 1.6 (dx = 0.1, five cells across the sheet half-width) with
    its 12^3 velocity grids: the FP32 form (FP32 f and sweeps, FP64 moment
    sums and fields, fitted) against the FP64 oracle over 12 steps. Each
    energy channel (kinetic+thermal of either species, electric, magnetic)
    agrees to 1e-5 of the total (the FP32 moment tolerance), and the total
    drifts by less than 1e-4 on both sides; the reconnected flux on the X
    line (the B_x null) agrees to 1e-6 and its change, the reconnection
    rate, to 1% of the oracle's."""
    from oracle.step import OracleState
    from paper_2109_06743_gb300.driver import Simulation
    cfg = W.asym_sheet(nx=32, ny=16, nv=12, lx=3.2, ly=1.6, precision=32)
    f = [x.astype(np.float32) for x in W.asym_state(cfg)]
    yee = W.asym_yee(cfg)
    yl = W.asym_null_y(cfg)
    sim = Simulation(cfg, f, None, yee)
    ost = OracleState(cfg, [x.astype(np.float64) for x in f], None, yee)
    psi0 = ost.reconnected_flux(yl)
    assert abs(sim.reconnected_flux(yl) - psi0) < 1e-15 * psi0 + 1e-300
    E0g, E0o = sim.total_energy(), ost.total_energy()
    steps = 12
    for _ in range(steps):
        sim.step()
        ost.step(cfg.dt)
    kg, eeg, ebg = sim.energies()
    ko, eeo, ebo = ost.energies()
    total = sum(ko) + eeo + ebo
    for a, b in zip(list(kg) + [eeg, ebg], list(ko) + [eeo, ebo]):
        assert abs(a - b) <= 1e-5 * total, (a, b, total)
    assert abs(total / E0o - 1) < 1e-4 and abs(sim.total_energy() / E0g - 1) < 1e-4
    pg, po = sim.reconnected_flux(yl), ost.reconnected_flux(yl)
    assert abs(pg - po) <= 1e-6 * po, (pg, po)
    rg, ro = (pg - psi0) / (steps * cfg.dt), (po - psi0) / (steps * cfg.dt)
    assert ro != 0.0 and abs(rg - ro) <= 1e-2 * abs(ro), (rg, ro)
    st = sim.stats()
    # boxes sized for the hot side: the device chose the wide fit kernel for
    # every fit, and no block needed the FP64-exponential evaluation
    assert st[3] == 0 and st[6] == 0 and st[9] == 2 * 2 * cfg.ncell * steps, st
    sim.close()
