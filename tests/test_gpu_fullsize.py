"""Parity at the benchmark's full sizes, in its launch configuration: the
Harris sheet 512 x 256 x 16^3 and the asymmetric sheet 1024 x 512 x 12^3
per species (its wide fit kernel), FP32, one step's passes issued
through the C ABI in the driver's order (fields, fused x+y sweep, velocity
pass with fused moments, fit, exchange). The oracle computes sampled
outputs one by one:

* fused x+y sweep: the value at a sampled (y, x, velocity) cell from the
  oracle's PFC line step along x of the rows y-4 .. y+4 (whole periodic
  lines) and then along y of those nine values (rows away from the
  walls), within 4e-6 of max f (two FP32 sweeps); over the whole grid, mass
  is conserved to 1e-6 and f stays non-negative;
* velocity pass: sampled blocks advected by the oracle with the cell's E and
  B, within 1e-5 of max f, and the fused moments within 1e-5 of their scale;
* fit: the fitted parameters of sampled cells (V and the rescaled F targets)
  equal the oracle's fits of the same targets to 1e-8;
* exchange: sampled blocks after the exchange equal the oracle's moment fit
  and exchange of the same block and fluid state within 2e-5 of max f;
* the fused sweep's edge tiles: samples in the four columns next to the
  periodic seam in x, and samples in the four rows next to either wall,
  whose oracle value comes from the oracle's PFC lines along x of the
  twelve rows next to the wall (the sampled velocity column and its v_y
  mirror) followed by the oracle's walled y sweep of those rows;
* the warm-started fit (use_mlp = 1, the benchmark's timed form) with a
  network trained as in the benchmark: fitted parameters of sampled cells
  equal the oracle's fits of the same targets to 1e-8.
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


@pytest.mark.parametrize("name", ["harris_512x256_v16", "asym_1024x512_v12"])
def test_full_size_passes_match_the_oracle_on_samples(gpu, orc, name):
    torch = gpu
    from paper_2109_06743_gb300 import abi
    from paper_2109_06743_gb300.driver import Simulation
    cfg = W.named(name, precision=32)
    f0 = W.initial_state(cfg, np.float32)
    sim = Simulation(cfg, f0, None, W.initial_yee(cfg))
    del f0
    ctx, s, dt, nv = sim.ctx, sim.stream, cfg.dt, cfg.species[0].nv[0]
    V = nv ** 3
    rng = np.random.default_rng(2109)
    abi.maxwell_step(ctx, 0.5 * dt, None, s)
    eb = None
    for k, sp in enumerate(cfg.species):
        g1 = orc.make_grid(3, 1, 1, 0.0, 1.0, 0.0, 1.0, 0)
        s1 = orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)
        # ---- fused x+y sweep ------------------------------------------------
        fin = sim.f[k].clone()
        mass0 = fin.double().sum().item()
        abi.pfc_advect_xy(ctx, k, dt, sim.f_spare[k], s)
        sim.f[k], sim.f_spare[k] = sim.f_spare[k], sim.f[k]
        torch.cuda.synchronize()
        fout = sim.f[k]
        assert abs(fout.double().sum().item() / mass0 - 1.0) < 1e-6
        assert fout.min().item() >= 0.0
        fin4 = fin.view(cfg.ny, cfg.nx, V)
        fmax = fin.max().item()
        vx, vy = sp.vcentres(0), sp.vcentres(1)
        for n_s in range(10):
            y, vi = int(rng.integers(8, cfg.ny - 8)), int(rng.integers(0, V))
            # the last four samples sit on the periodic seam in x
            x = int(rng.integers(0, cfg.nx)) if n_s < 6 else [0, 1, cfg.nx - 2, cfg.nx - 1][n_s - 6]
            ix, iy = vi % nv, (vi // nv) % nv
            cx, cy = vx[ix] * dt / cfg.dx, vy[iy] * dt / cfg.dy
            assert abs(cx) < 1 and abs(cy) < 1
            rows = fin4[y - 4:y + 5, :, vi].double().cpu().numpy()
            xs = np.array([orc.pfc_line(np.concatenate([r[-4:], r, r[:4]]), cfg.nx, 4, cx)[x] for r in rows])
            want = orc.pfc_line(xs, 1, 4, cy)[0]
            got = fout.view(cfg.ny, cfg.nx, V)[y, x, vi].item()
            assert abs(got - want) <= 4e-6 * fmax, (k, y, x, vi, got, want)
        # rows next to the walls: x sweeps of the 12 rows nearest the wall for
        # the sampled column and its v_y mirror (the wall's ghost column), then
        # the oracle's walled y sweep of those rows
        gw = orc.make_grid(3, 1, 12, 0.0, cfg.dx, 0.0, cfg.dy, 1)
        for n_s in range(4):
            x, vi = int(rng.integers(0, cfg.nx)), int(rng.integers(0, V))
            ix, iy, iz = vi % nv, (vi // nv) % nv, vi // (nv * nv)
            vm = (iz * nv + (nv - 1 - iy)) * nv + ix
            cx = vx[ix] * dt / cfg.dx
            top = n_s % 2 == 1
            rows = list(range(cfg.ny - 12, cfg.ny)) if top else list(range(12))
            sub = np.zeros((12, V))
            for col in (vi, vm):
                lines = fin4[rows[0]:rows[-1] + 1, :, col].double().cpu().numpy()
                for jr, r in enumerate(lines):
                    sub[jr, col] = orc.pfc_line(np.concatenate([r[-4:], r, r[:4]]), cfg.nx, 4, cx)[x]
            # the sub-grid has walls at both ends; only the one next to the
            # checked rows is the workload's
            orc.advect_space(sub, gw, s1, 1, dt)
            for jr in ((8, 9, 10, 11) if top else (0, 1, 2, 3)):
                got = fout.view(cfg.ny, cfg.nx, V)[rows[jr], x, vi].item()
                assert abs(got - sub[jr, vi]) <= 4e-6 * fmax, (k, rows[jr], x, vi, got, sub[jr, vi])
        # ---- velocity pass with fused moments --------------------------------
        cells = rng.integers(0, cfg.ncell, 6)
        ct = torch.as_tensor(cells, device=sim.dev)
        before = fout[ct].double().cpu().numpy()
        abi.pfc_advect_v(ctx, k, dt, sim.mom_t1[k], s)
        torch.cuda.synchronize()
        eb = sim.eb.cpu().numpy()
        after = sim.f[k][ct].double().cpu().numpy()
        mom = sim.mom_t1[k][ct].cpu().numpy()
        for j, c in enumerate(cells):
            ref = np.ascontiguousarray(before[j:j + 1]).copy()
            orc.advect_velocity(ref, g1, s1, np.ascontiguousarray(eb[c:c + 1]), dt, 5)
            assert np.abs(after[j] - ref[0]).max() <= 1e-5 * fmax
            m_ref = orc.moments(np.ascontiguousarray(after[j:j + 1]), g1, s1)[0]
            v = [np.abs(sp.vcentres(a)) for a in range(3)]
            fb = np.abs(after[j]).reshape(nv, nv, nv)
            dv3 = float(np.prod(sp.dv))
            scale = np.array([np.einsum("zyx,x,y,z->", fb, v[0] ** a, v[1] ** b, v[2] ** c_) * dv3
                              for a, b, c_ in W_MONO]) + 1e-300
            assert np.all(np.abs(mom[j] - m_ref) <= 1e-5 * scale)
    # ---- fluid, fit and exchange (species 0 and 1) ---------------------------
    abi.fluid_step(ctx, dt, sim.mom_t, sim.mom_t1, s)
    torch.cuda.synchronize()
    for k, sp in enumerate(cfg.species):
        g1 = orc.make_grid(3, 1, 1, 0.0, 1.0, 0.0, 1.0, 0)
        s1 = orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)
        cells = rng.integers(0, cfg.ncell, 4)
        ct = torch.as_tensor(cells, device=sim.dev)
        fluid_before = sim.fluid[k][ct].cpu().numpy().copy()
        f_before = sim.f[k][ct].double().cpu().numpy()
        fmax = sim.f[k].max().item()
        thv = torch.zeros((cfg.ncell, 10), dtype=torch.float64, device=sim.dev)
        thf = torch.zeros_like(thv)
        abi.moment_fit_solve(ctx, k, sim.mom_t1[k], False, thv, thf, s)
        abi.moment_fit_exchange(ctx, k, sim.mom_t1[k], sim.mom_t[k], s)
        torch.cuda.synchronize()
        vm = sim.mom_t1[k][ct].cpu().numpy()
        fl = sim.fluid[k][ct].cpu().numpy()
        f_after = sim.f[k][ct].double().cpu().numpy()
        for j, c in enumerate(cells):
            tv, it, st = orc.maxent_fit(vm[j, :10], s1, 3, cfg.fit_tol, cfg.fit_max_iter)
            assert st == 0
            np.testing.assert_allclose(thv[c].cpu().numpy(), tv, rtol=1e-8, atol=1e-12 * abs(tv).max())
            tf, it, st = orc.maxent_fit(fl[j], s1, 3, cfg.fit_tol, cfg.fit_max_iter)
            assert st == 0
            np.testing.assert_allclose(thf[c].cpu().numpy(), tf, rtol=1e-8, atol=1e-12 * abs(tf).max())
            ref = np.ascontiguousarray(f_before[j:j + 1]).copy()
            U = np.ascontiguousarray(fluid_before[j:j + 1]).copy()
            orc.moment_fit(ref, g1, s1, U, cfg.fit_tol, cfg.fit_max_iter)
            assert np.abs(f_after[j] - ref[0]).max() <= 2e-5 * fmax
    st = abi.vl_read_stats(ctx)
    assert st[8] == 0
    # the fit kernel chosen on the device: the wide one for the asymmetric
    # sheet (boxes sized for its hot side), the common one for the Harris
    # sheet; no FP64-exponential evaluations either way
    assert st[9] == (2 * cfg.ncell if cfg.kind == "asym" else 0) * 2 and st[6] == 0, st
    # ---- the warm-started fit (use_mlp = 1, the benchmark's timed form) -------
    from paper_2109_06743_gb300.warmstart import train_warm_start
    w, _ = train_warm_start(W.TRAIN_FROM[name], sim.dev)
    abi.mlp_set_weights(ctx, w)
    abi.vl_reset_stats(ctx, s)
    for k, sp in enumerate(cfg.species):
        s1 = orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)
        cells = rng.integers(0, cfg.ncell, 4)
        ct = torch.as_tensor(cells, device=sim.dev)
        thv = torch.zeros((cfg.ncell, 10), dtype=torch.float64, device=sim.dev)
        thf = torch.zeros_like(thv)
        abi.moment_fit_solve(ctx, k, sim.mom_t1[k], True, thv, thf, s)
        torch.cuda.synchronize()
        vm = sim.mom_t1[k][ct].cpu().numpy()
        fl = sim.fluid[k][ct].cpu().numpy()
        for j, c in enumerate(cells):
            for targets, th_gpu in ((vm[j, :10], thv[c]), (fl[j], thf[c])):
                th, it, st_ = orc.maxent_fit(np.ascontiguousarray(targets), s1, 3, cfg.fit_tol, cfg.fit_max_iter)
                assert st_ == 0
                np.testing.assert_allclose(th_gpu.cpu().numpy(), th, rtol=1e-8, atol=1e-12 * abs(th).max())
    st = abi.vl_read_stats(ctx, s)
    assert st[12] > 0.9 * 2 * cfg.ncell * len(cfg.species) and st[1] == 0, st  # started from the network
    sim.close()


W_MONO = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1),
          (0, 0, 2), (3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1),
          (0, 1, 2), (0, 0, 3)]
