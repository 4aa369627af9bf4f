"""The limiter of the exchange (Algorithm 1's moment fitting, Sec. 2.2) on
the GPU against the oracle: where f - M_V + M_F has negative values, the
cell's block is clipped at zero and rescaled to the density n_V of the
targets it was fitted to; cells without negative values are left as the
exchange made them.

Each cell's f is one sampled Maxwellian well inside the velocity box (so
that f - M_V + M_F keeps a wide positive margin where nothing is done to
it) times 1 +- 5% noise. Every fifth spatial cell gets
holes (every seventh velocity cell at 0.2 of its value) and fluid targets
whose mean sits 1.5 dv away and whose temperature is 0.7 of the kinetic
one, so that the exchange goes negative there by a large margin (the FP32
and FP64 sides take the same clipping decision); the other cells keep the
small fluid mismatch of the other parity tests, which clips a few of them
where the shifted tails reach below f (by a few per cent of the local
values, again the same decision on both sides). Compared: f after the exchange
element by element (1e-10 of max f in FP64, 2e-5 in FP32, as the fit
tests), the number of clipped cells, the fused moments of the new f, the
density n_V kept in the clipped cells and f >= 0.
"""
import numpy as np
import pytest

from paper_2109_06743_gb300 import workloads as W
from test_gpu_kernels import cast, fluid_targets, oracle_grid, oracle_species

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2109_06743_gb300 import build
    build.build()
    return torch


def maxwellian_cells(cfg, orc, seed, pert=0.05):
    """per cell, a sampled Maxwellian well inside the velocity box (n in
    [0.5, 1.5], |u_a| <= dv, Theta_aa = (1.2 dv)^2 [0.8, 1.2], correlation
    coefficients up to 0.1), times 1 +- pert noise"""
    rng = np.random.default_rng(seed)
    out = []
    for sp in cfg.species:
        s = oracle_species(orc, sp)
        dv = np.array(sp.dv)
        blocks = []
        for c in range(cfg.ncell):
            n = rng.uniform(0.5, 1.5)
            u = dv * rng.uniform(-1, 1, 3)
            sd = 1.2 * dv * np.sqrt(rng.uniform(0.8, 1.2, 3))
            r = 0.1 * rng.uniform(-1, 1, 3)
            th = [sd[0] ** 2, r[0] * sd[0] * sd[1], r[1] * sd[0] * sd[2], sd[1] ** 2, r[2] * sd[1] * sd[2], sd[2] ** 2]
            M = orc.maxwellian_grid(np.concatenate([[n], u, th]), s, 3)
            blocks.append(M * (1.0 + pert * rng.uniform(-1, 1, M.size)))
        out.append(np.ascontiguousarray(np.stack(blocks)))
    return out


def _raw(n, u, th):
    uu = np.outer(u, u)
    P = n * (th + uu)
    return np.array([n, n * u[0], n * u[1], n * u[2], P[0, 0], P[0, 1], P[0, 2], P[1, 1], P[1, 2], P[2, 2]])


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("nv", [12, 16])
def test_exchange_limiter_matches_oracle(gpu, orc, precision, nv):
    from gpu_util import AbiRunner
    from paper_2109_06743_gb300 import abi
    cfg = W.harris(nx=5, ny=4, nv=nv, lx=1.0, ly=0.8, precision=precision)
    cfg.fit_tol = 1e-12
    f0 = maxwellian_cells(cfg, orc, 930)
    holes = np.arange(cfg.ncell) % 5 == 0
    for f in f0:
        f[np.ix_(holes, np.arange(0, f.shape[1], 7))] *= 0.2
    f0 = [cast(np.ascontiguousarray(f), precision) for f in f0]
    U0 = fluid_targets(cfg, orc, f0, 931)
    g = oracle_grid(orc, cfg)
    for k, sp in enumerate(cfg.species):
        m = orc.moments(f0[k], g, oracle_species(orc, sp))
        dv = np.array(sp.dv)
        for c in np.nonzero(holes)[0]:
            n = m[c, 0]
            u = m[c, 1:4] / n
            E2 = m[c, 4:10] / n
            th = np.array([[E2[0], E2[1], E2[2]], [E2[1], E2[3], E2[4]], [E2[2], E2[4], E2[5]]]) - np.outer(u, u)
            U0[k][c] = _raw(n, u + np.array([1.5 * dv[0], 0.0, 0.0]), 0.7 * th)
    r = AbiRunner(cfg, f0, fluid=np.stack(U0))
    for k, sp in enumerate(cfg.species):
        s = oracle_species(orc, sp)
        vmom = r.mom()
        abi.moments(r.ctx, k, vmom)
        mout = r.mom()
        abi.vl_reset_stats(r.ctx)
        abi.moment_fit(r.ctx, k, vmom, False, None, None, mout)
        st_gpu = abi.vl_read_stats(r.ctx)
        ref_f = f0[k].copy()
        ref_U = U0[k].copy()
        nV = orc.moments(ref_f, g, s)[:, 0].copy()
        st = orc.moment_fit(ref_f, g, s, ref_U, cfg.fit_tol, cfg.fit_max_iter)
        # every holed cell is clipped, and the GPU clips as many cells as the oracle
        assert st[2] >= int(holes.sum()) and st_gpu[2] == st[2], (st, st_gpu)
        assert st_gpu[1] == st[1] and st_gpu[3] == 0, (st, st_gpu)
        got = r.f_np(k)
        tol = (1e-10 if precision == 64 else 2e-5) * ref_f.max()
        assert np.abs(got - ref_f).max() <= tol, (np.abs(got - ref_f).max(), tol)
        assert got.min() >= 0.0
        # the fused moments of the new f, and the density kept in clipped cells
        mref = orc.moments(ref_f, g, s)
        mg = mout.cpu().numpy()
        n_ = mref[:, :1]
        scale = np.concatenate([n_, n_ * dv.max() * np.ones((1, 3)), n_ * dv.max() ** 2 * np.ones((1, 6))], axis=1)
        rel = 1e-10 if precision == 64 else 2e-5
        assert np.all(np.abs(mg[:, :10] - mref[:, :10]) <= rel * scale), float(np.max(np.abs(mg[:, :10] - mref[:, :10]) / scale))
        np.testing.assert_allclose(mg[holes, 0], nV[holes], rtol=1e-12 if precision == 64 else 2e-6)
    r.close()
