"""The Newton fit's arithmetic and kernel choice behind the C ABI (paper
Sec. 2.2, Algorithm 1's moment fitting), and the device status word.

* FP64 mode fits in plain FP64 arithmetic (fit tolerance 1e-13 n on both
  sides). The GPU's fitted Maxwellians, evaluated on the grid by the
  oracle's own definition (or_maxwellian_grid, then or_moments), reproduce
  the targets to 1e-12 of their scale: the defining property of the
  discrete fit. Their parameters equal the oracle's fit of the same
  targets to 1e-12 relative on the 12^3 to 24^3 grids; the two sides differ
  only in the order of roundings (both evaluate the moments to about
  1e-15), which the Jacobian's conditioning amplifies on 8^3 blocks, where
  the ions' Maxwellians span little more than one velocity cell per
  thermal speed: 1e-10 there. Where every fit converges, the total Newton
  iteration count equals the oracle's (the same iteration: start, Jacobian,
  damping rule), and the
  exchanged f equals the oracle's moment fit to 1e-11 of max f. Block sizes
  8-24, the Harris sheet and the narrow Maxwellians of the asymmetric
  sheet.
* FP32 mode chooses between its two double-float kernels on the device:
  with no moment_fit_wide call the asymmetric sheet's cells (Maxwellians
  narrow against velocity boxes sized for the hot side) are fitted by the
  wide kernel with no FP64-exponential evaluation, the Harris sheet's by
  the common one.
* A non-finite or negative fit target sets the status word: the next
  compute call returns VL_ENUMERIC without enqueueing work, and
  vl_sync_status reports it too; empty cells (n = 0) are no error.
"""
import numpy as np
import pytest

from paper_2109_06743_gb300 import workloads as W
from test_gpu_kernels import cast, fluid_targets, near_maxwellian_state, oracle_grid, oracle_species

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2109_06743_gb300 import build
    build.build()
    return torch


def _fit_against_oracle(r, cfg, orc, f0, U0, check_iters=True, theta_tol=1e-12):
    from paper_2109_06743_gb300 import abi
    g = oracle_grid(orc, cfg)
    g1 = orc.make_grid(3, 1, 1, 0.0, 1.0, 0.0, 1.0, 0)
    for k, sp in enumerate(cfg.species):
        s = oracle_species(orc, sp)
        vmom = r.mom()
        abi.moments(r.ctx, k, vmom)
        thv = r.torch.zeros((cfg.ncell, 10), dtype=r.torch.float64, device=r.dev)
        thf = r.torch.zeros_like(thv)
        abi.moment_fit(r.ctx, k, vmom, False, thv, thf, None)
        r.sync()
        ref_f = f0[k].copy()
        ref_U = U0[k].copy()
        st = orc.moment_fit(ref_f, g, s, ref_U, cfg.fit_tol, cfg.fit_max_iter)
        got = r.f_np(k)
        f_err = np.abs(got - ref_f).max() / ref_f.max()
        vm = vmom.cpu().numpy()
        fl = r.fluid[k].cpu().numpy()
        tv, tf = thv.cpu().numpy(), thf.cpu().numpy()
        worst, resid = 0.0, 0.0
        for c in range(cfg.ncell):
            for targets, got_th in ((vm[c, :10], tv[c]), (fl[c], tf[c])):
                th, it, stt = orc.maxent_fit(np.ascontiguousarray(targets), s, 3, cfg.fit_tol, cfg.fit_max_iter)
                if stt == 0:
                    # n', u' and Theta' against their own scales
                    sc = np.array([th[0]] + [np.sqrt(th[4] + th[7] + th[9])] * 3 + [th[4] + th[7] + th[9]] * 6)
                    worst = max(worst, float(np.max(np.abs(got_th - th) / sc)))
                    # the GPU's Maxwellian on the grid, by the oracle's definition
                    fm = orc.maxwellian_grid(got_th, s, 3).reshape(1, -1)
                    mm = orc.moments(np.ascontiguousarray(fm), g1, s)[0, :10]
                    n = targets[0]
                    v2 = np.sqrt((targets[4] + targets[7] + targets[9]) / n)
                    msc = n * np.array([1.0, v2, v2, v2] + [v2 * v2] * 6)
                    resid = max(resid, float(np.max(np.abs(mm - targets) / msc)))
        assert resid <= 1e-12 and worst <= theta_tol and f_err <= 1e-11, (resid, worst, f_err)
        stats = abi.vl_read_stats(r.ctx)
        assert stats[1] == st[1] and stats[3] == 0, (stats, st)
        if check_iters and st[1] == 0:
            # (fits that do not converge may give up at different iterations)
            assert stats[0] == st[0], (stats[0], st[0])
        # every fit by the FP64 kernel
        assert stats[10] > 0 and stats[4] == 0 and stats[6] == 0, stats
        abi.vl_reset_stats(r.ctx)


@pytest.mark.parametrize("nv", [8, 12, 16, 20, 24])
def test_fp64_fit_matches_oracle_to_1e12(gpu, orc, nv):
    from gpu_util import AbiRunner
    cfg = W.harris(nx=6, ny=6 if nv <= 16 else 3, nv=nv, lx=25.6 * 6 / 128, ly=12.8 * 6 / 64, precision=64)
    cfg.bc_y = 1
    cfg.fit_tol = 1e-13
    f0 = near_maxwellian_state(cfg, 400 + nv)
    U0 = fluid_targets(cfg, orc, f0, 401 + nv)
    r = AbiRunner(cfg, f0, fluid=np.stack(U0))
    _fit_against_oracle(r, cfg, orc, f0, U0, theta_tol=1e-12 if nv >= 12 else 1e-10)
    r.close()


def test_fp64_fit_of_narrow_maxwellians_matches_oracle(gpu, orc):
    from gpu_util import AbiRunner
    cfg = W.asym_sheet(nx=3, ny=16, nv=12, lx=0.6, ly=6.4, precision=64)
    cfg.fit_tol = 1e-13
    rng = np.random.default_rng(412)
    f0 = [np.ascontiguousarray(f.reshape(cfg.ncell, -1) * (1.0 + 0.05 * rng.uniform(-1, 1, (cfg.ncell, 1))))
          for f in W.asym_state(cfg)]
    U0 = fluid_targets(cfg, orc, f0, 413)
    r = AbiRunner(cfg, f0, fluid=np.stack(U0))
    _fit_against_oracle(r, cfg, orc, f0, U0)
    r.close()


@pytest.mark.parametrize("kind", ["asym", "harris"])
def test_fp32_fit_kernel_is_chosen_on_the_device(gpu, orc, kind):
    from gpu_util import AbiRunner
    from paper_2109_06743_gb300 import abi
    if kind == "asym":
        cfg = W.asym_sheet(nx=4, ny=16, nv=12, lx=0.8, ly=6.4, precision=32)
        f0 = [cast(f.reshape(cfg.ncell, -1), 32) for f in W.asym_state(cfg)]
    else:
        cfg = W.harris(nx=8, ny=16, nv=12, precision=32)  # the full 25.6 x 12.8 box
        f0 = [cast(f.reshape(cfg.ncell, -1), 32) for f in W.harris_state(cfg)]
    U0 = fluid_targets(cfg, orc, f0, 414)
    r = AbiRunner(cfg, f0, fluid=np.stack(U0))
    thv = r.torch.zeros((cfg.ncell, 10), dtype=r.torch.float64, device=r.dev)
    g = oracle_grid(orc, cfg)
    for k, sp in enumerate(cfg.species):
        vmom = r.mom()
        abi.moments(r.ctx, k, vmom)
        abi.moment_fit(r.ctx, k, vmom, False, thv, None, None)
        st = abi.vl_read_stats(r.ctx)
        if kind == "asym":
            assert st[9] == 2 * cfg.ncell and st[6] == 0 and st[4] > 0, st
        else:
            assert st[9] == 0 and st[6] == 0 and st[4] > 0, st
        vm = vmom.cpu().numpy()
        s = oracle_species(orc, sp)
        for c in range(0, cfg.ncell, 5):
            th, it, stt = orc.maxent_fit(vm[c, :10], s, 3, cfg.fit_tol, cfg.fit_max_iter)
            if stt == 0:
                np.testing.assert_allclose(thv[c].cpu().numpy(), th, rtol=1e-8, atol=1e-12 * abs(th).max())
        abi.vl_reset_stats(r.ctx)
    r.close()


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("where", ["moments", "fluid"])
def test_nonfinite_targets_are_reported_by_the_next_call(gpu, orc, precision, where):
    from gpu_util import AbiRunner
    from paper_2109_06743_gb300 import abi
    cfg = W.harris(nx=4, ny=4, nv=8, lx=0.8, ly=0.8, precision=precision)
    f0 = [cast(f, precision) for f in near_maxwellian_state(cfg, 702)]
    U0 = np.stack(fluid_targets(cfg, orc, f0, 703))
    r = AbiRunner(cfg, f0, fluid=U0)
    vm = r.mom()
    abi.moments(r.ctx, 0, vm)
    # a clean fit leaves the word clear; so does an empty cell (n = 0)
    abi.moment_fit(r.ctx, 0, vm, False, None, None, None)
    abi.vl_sync_status(r.ctx)
    vm[5] = 0.0
    r.fluid[0, 5] = 0.0
    abi.moment_fit(r.ctx, 0, vm, False, None, None, None)
    abi.vl_sync_status(r.ctx)
    abi.moments(r.ctx, 0, vm)
    if where == "moments":
        vm[3, 4] = float("nan")
    else:
        r.fluid[0, 3, 0] = -1.0
    abi.moment_fit_solve(r.ctx, 0, vm, False, None, None)
    r.sync()
    # the next compute call reports it and enqueues nothing
    before = r.f[1].clone()
    with pytest.raises(abi.VlasovError) as e:
        abi.pfc_advect_v(r.ctx, 1, 0.01, None)
    assert e.value.status == abi.VL_ENUMERIC
    r.sync()
    assert r.torch.equal(before, r.f[1])
    # reported once: the following call runs
    abi.pfc_advect_v(r.ctx, 1, 0.01, None)
    abi.vl_sync_status(r.ctx)
    # and vl_sync_status reports an error found by the last call (the fit
    # replaced the fluid state by its rescaled moments: plant the error again)
    if where == "fluid":
        r.fluid[0, 3, 0] = -1.0
    abi.moment_fit_solve(r.ctx, 0, vm, False, None, None)
    with pytest.raises(abi.VlasovError) as e:
        abi.vl_sync_status(r.ctx)
    assert e.value.status == abi.VL_ENUMERIC
    abi.vl_sync_status(r.ctx)
    r.close()
