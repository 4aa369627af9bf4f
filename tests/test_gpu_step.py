"""GPU parity of whole time steps (Algorithm 1, paper Sec. 2.2) through the
C-ABI against the FP64 oracle, and the physics pins of Sec. 3.1 on the GPU.

* FP64 Harris sheet (walls in y, CFL < 1) and a periodic smooth wave: f,
  fluid state and fields after a few steps agree with the oracle to 1e-10
  relative (FP64 throughout; differences are rounding order only).
* FP32 Harris sheet: f within 2e-5 max|f| after 3 steps, total energy
  within 1e-6 relative of the oracle's (energy drift parity; the FP32-mode
  drift tolerance is 1e-4).
* Linear Landau damping on the GPU path (FP64): damping rate and frequency
  within 1% of the dispersion root, mass to 1e-12, energy to 1e-5, and the
  E(t) history equal to the oracle's to 1e-9.
"""
import math

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


def run_both(cfg, f, yee, steps):
    from oracle.step import OracleState
    from paper_2109_06743_gb300.driver import Simulation
    ost = OracleState(cfg, f, None, yee)
    sim = Simulation(cfg, f, None, yee)
    for _ in range(steps):
        ost.step(cfg.dt)
        sim.step()
    return ost, sim


@pytest.mark.parametrize("kind", ["harris", "wave"])
def test_fp64_steps_match_oracle(gpu, orc, kind):
    if kind == "harris":
        cfg = W.harris(nx=16, ny=8, nv=8, lx=3.2, ly=1.6, precision=64)
        f, yee = W.harris_state(cfg), W.harris_yee(cfg)
    else:
        cfg = W.wave2d(nx=12, ny=6, nv=8, precision=64)
        f, yee = W.wave2d_state(cfg), W.wave2d_yee(cfg)
    cfg.fit_tol = 1e-12
    ost, sim = run_both(cfg, f, yee, 3)
    for k in range(2):
        ref = ost.f[k]
        got = sim.f_host(k)
        assert np.abs(got - ref).max() <= 1e-10 * ref.max(), np.abs(got - ref).max() / ref.max()
        np.testing.assert_allclose(sim.fluid[k].cpu().numpy(), ost.U[k], rtol=1e-10,
                                   atol=1e-12 * np.abs(ost.U[k]).max())
    np.testing.assert_allclose(sim.yee.cpu().numpy(), ost.yee, rtol=0, atol=1e-10 * np.abs(ost.yee).max())
    st = sim.stats()
    assert st[1] == 0 and st[3] == 0
    # FP64 mode: every fit by the plain FP64 kernel
    assert st[10] > 0 and st[4] == 0 and st[9] == 0, st
    sim.close()


def test_fp32_steps_match_oracle(gpu, orc):
    cfg = W.harris(nx=16, ny=8, nv=8, lx=3.2, ly=1.6, precision=32)
    f = [x.astype(np.float32).astype(np.float64) for x in W.harris_state(cfg)]
    yee = W.harris_yee(cfg)
    ost, sim = run_both(cfg, f, yee, 3)
    for k in range(2):
        ref = ost.f[k]
        got = sim.f_host(k)
        assert np.abs(got - ref).max() <= 2e-5 * ref.max(), np.abs(got - ref).max() / ref.max()
    e_or = ost.total_energy()
    e_gpu = sim.total_energy()
    assert abs(e_gpu - e_or) <= 1e-6 * e_or, (e_gpu, e_or)
    sim.close()


def test_landau_damping_on_gpu(gpu, orc):
    from oracle.step import OracleState
    from paper_2109_06743_gb300.driver import Simulation
    from test_oracle_physics import dispersion_root, rate_and_frequency
    cfg = W.landau()
    f0 = W.landau_state(cfg)
    sim = Simulation(cfg, f0)
    ost = OracleState(cfg, f0)
    x = cfg.x0 + (np.arange(cfg.nx) + 0.5) * cfg.dx
    E0 = sim.total_energy()
    m0 = f0[0].sum()
    ts, amps, maxdiff = [], [], 0.0
    for n in range(cfg.steps):
        sim.step()
        ost.step(cfg.dt)
        e = sim.eb[:, 0].cpu().numpy()
        maxdiff = max(maxdiff, np.abs(e - ost.EB[:, 0]).max())
        ts.append(sim.time)
        amps.append(2 * abs(np.sum(e * np.exp(-1j * cfg.k * x))) / cfg.nx)
    wr, wi = dispersion_root(cfg.k)
    gamma, omega = rate_and_frequency(np.array(ts), np.array(amps))
    assert abs(gamma - wi) / abs(wi) < 0.01
    assert abs(omega - wr) / wr < 0.01
    assert maxdiff < 1e-9
    assert abs(sim.f_host(0).sum() - m0) <= 1e-12 * m0
    assert abs(sim.total_energy() - E0) <= 1e-5 * E0
    sim.close()


def test_asymmetric_sheet_fp64_steps_match_oracle(gpu, orc):
    """The asymmetric (magnetopause-like) sheet, downscaled: density ratio 10,
    temperature ratio 3, guide field 0.1, m_i/m_e = 100; FP64 steps equal
    the oracle's to 1e-10."""
    cfg = W.asym_sheet(nx=16, ny=16, nv=8, lx=3.2, ly=6.4, precision=64)
    cfg.fit_tol = 1e-12
    f, yee = W.asym_state(cfg), W.asym_yee(cfg)
    ost, sim = run_both(cfg, f, yee, 2)
    for k in range(2):
        ref = ost.f[k]
        got = sim.f_host(k)
        assert np.abs(got - ref).max() <= 1e-10 * ref.max(), np.abs(got - ref).max() / ref.max()
    np.testing.assert_allclose(sim.yee.cpu().numpy(), ost.yee, rtol=0, atol=1e-10 * np.abs(ost.yee).max())
    assert sim.stats()[3] == 0
    sim.close()


@pytest.mark.parametrize("fit", [True, False])
def test_step_through_host_equals_device_steps(gpu, fit):
    """The end-to-end form (f copied in from and out to pinned host buffers
    every step, the copies on their own streams overlapping the other
    species' kernels) gives bit for bit the f of the same steps run on the
    device."""
    from paper_2109_06743_gb300.driver import Simulation
    torch = gpu
    cfg = W.harris(nx=32, ny=16, nv=8, lx=6.4, ly=3.2)
    f0 = W.harris_state(cfg, dtype=np.float32)
    a = Simulation(cfg, f0, None, W.harris_yee(cfg), fit=fit)
    b = Simulation(cfg, f0, None, W.harris_yee(cfg), fit=fit)
    host = [torch.empty(f.shape, dtype=f.dtype, pin_memory=True) for f in b.f]
    for h, f in zip(host, b.f):
        h.copy_(f)
    for _ in range(4):
        a.step()
        b.step_through_host(host)
    b.wait_host()
    torch.cuda.synchronize()
    for k in range(2):
        assert torch.equal(host[k], a.f[k].cpu())
    a.close()
    b.close()


@pytest.mark.parametrize("kind", ["landau", "harris"])
def test_graph_replay_equals_launched_steps(gpu, kind):
    """Steps captured once in a CUDA graph and replayed give bit for bit the
    f of the same steps launched one by one (1D1V Landau; 2D3V Harris with
    the fused sweep's buffer swap over an even number of steps)."""
    from paper_2109_06743_gb300.driver import Simulation
    torch = gpu
    if kind == "landau":
        cfg = W.landau()
        f0 = W.landau_state(cfg)
        yee = None
    else:
        cfg = W.harris(nx=32, ny=16, nv=8, lx=6.4, ly=3.2)
        f0 = W.harris_state(cfg, dtype=np.float32)
        yee = W.harris_yee(cfg)
    a = Simulation(cfg, f0, None, yee)
    b = Simulation(cfg, f0, None, yee, stream=torch.cuda.Stream())
    a.step()
    b.step()
    g = b.graph(4)
    for _ in range(8):
        a.step()
    with torch.cuda.stream(b.stream):
        g.replay()
        g.replay()
    torch.cuda.synchronize()
    for k in range(len(cfg.species)):
        assert torch.equal(a.f[k], b.f[k])
    a.close()
    b.close()
