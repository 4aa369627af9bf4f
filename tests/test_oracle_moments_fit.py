"""Pins of the oracle's moments (paper Sec. 2.1), the discrete ten-moment
Maxwellian fit and the exchange step of moment fitting (Sec. 2.2, Algorithm 1).

What fixes them:
* moments of a separable f factorise into products of 1D sums (independent
  evaluation); a finely sampled Maxwellian has moments (n, u, T) and zero
  heat flux (closed form, spectral accuracy of the midpoint rule); the heat
  flux relation Q = Qcal - sym(u x P) + 2 m n u u u equals the central third
  moment m int (v-u)^3 f.
* the fitted Maxwellian, sampled with the paper's formula and summed by
  numpy, reproduces the targets; on fine grids the fit tends to the targets;
  a 1D fit agrees with scipy root finding from a different start;
  infeasible targets fall back to the continuous Maxwellian.
* exchange: without clipping, the moments after the exchange are the fluid
  targets ("exact recovery of n, u, T"); density is n_V to rounding with or
  without clipping; f >= 0; a Maxwellian f with V = F is unchanged.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2109_06743_gb300 import workloads as W

MONO = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1),
        (0, 0, 2), (3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1),
        (0, 1, 2), (0, 0, 3)]


def box(nv, vm, q=1.0, m=1.0, name="s"):
    return W.SpeciesCfg(name, q, m, (nv, nv, nv), (-vm,) * 3, (vm,) * 3)


def orc_species(orc, sp):
    return orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)


def test_moments_separable(orc):
    sp = W.SpeciesCfg("s", 1.0, 1.0, (6, 5, 4), (-1.0, -2.0, -0.5), (2.0, 1.0, 1.5))
    g = orc.make_grid(3, 1, 1, 0.0, 1.0, 0.0, 1.0, 0)
    a = W.random_blocks(6, 1)
    b = W.random_blocks(5, 2)
    c = W.random_blocks(4, 3)
    f = (c[:, None, None] * b[None, :, None] * a[None, None, :]).reshape(1, -1)
    mom = orc.moments(np.ascontiguousarray(f), g, orc_species(orc, sp))[0]
    v = [sp.vcentres(k) for k in range(3)]
    dv = sp.dv
    for k, (p, q, r) in enumerate(MONO):
        ref = (np.sum(a * v[0] ** p) * dv[0]) * (np.sum(b * v[1] ** q) * dv[1]) * (np.sum(c * v[2] ** r) * dv[2])
        assert abs(mom[k] - ref) <= 1e-13 * max(1.0, abs(ref))


def sampled_maxwellian(sp, n, u, Th):
    v = [sp.vcentres(k) for k in range(3)]
    VZ, VY, VX = np.meshgrid(v[2], v[1], v[0], indexing="ij")
    d = np.stack([VX - u[0], VY - u[1], VZ - u[2]], axis=-1)
    Ti = np.linalg.inv(Th)
    q = np.einsum("...a,ab,...b->...", d, Ti, d)
    return n * (2 * math.pi) ** -1.5 / math.sqrt(np.linalg.det(Th)) * np.exp(-0.5 * q)


def test_fine_maxwellian_moments_and_heat_flux(orc):
    sp = box(48, 9.0)
    g = orc.make_grid(3, 1, 1, 0.0, 1.0, 0.0, 1.0, 0)
    n, u = 1.3, np.array([0.4, -0.3, 0.2])
    Th = np.array([[1.0, 0.2, -0.1], [0.2, 0.8, 0.05], [-0.1, 0.05, 1.2]])
    f = sampled_maxwellian(sp, n, u, Th).reshape(1, -1)
    mom = orc.moments(np.ascontiguousarray(f), g, orc_species(orc, sp))[0]
    assert abs(mom[0] - n) < 1e-12
    np.testing.assert_allclose(mom[1:4] / mom[0], u, atol=1e-12)
    E2 = np.array([[mom[4], mom[5], mom[6]], [mom[5], mom[7], mom[8]], [mom[6], mom[8], mom[9]]])
    np.testing.assert_allclose(E2 / n - np.outer(u, u), Th, atol=1e-11)
    # heat flux from the paper's relation (m = 1) vs the central third moment
    idx3 = {}
    for k, (p, q, r) in enumerate(MONO[10:]):
        idx3[(p, q, r)] = mom[10 + k]

    def Qcal(i, j, k):
        c = [0, 0, 0]
        for a in (i, j, k):
            c[a] += 1
        return idx3[tuple(c)]

    P = E2
    for i, j, k in itertools.product(range(3), repeat=3):
        Q = Qcal(i, j, k) - (u[i] * P[j, k] + u[j] * P[i, k] + u[k] * P[i, j]) + 2 * n * u[i] * u[j] * u[k]
        assert abs(Q) < 1e-10, (i, j, k, Q)


def test_heat_flux_relation_equals_central_moment(orc):
    sp = box(8, 3.0)
    g = orc.make_grid(3, 1, 1, 0.0, 1.0, 0.0, 1.0, 0)
    f = W.random_blocks((1, 512), 4)
    mom = orc.moments(f, g, orc_species(orc, sp))[0]
    n = mom[0]
    u = mom[1:4] / n
    P = np.array([[mom[4], mom[5], mom[6]], [mom[5], mom[7], mom[8]], [mom[6], mom[8], mom[9]]])
    v = [sp.vcentres(k) for k in range(3)]
    VZ, VY, VX = np.meshgrid(v[2], v[1], v[0], indexing="ij")
    V = [VX.ravel() - u[0], VY.ravel() - u[1], VZ.ravel() - u[2]]
    dv3 = np.prod(sp.dv)
    mono3 = {m: mom[10 + k] for k, m in enumerate(MONO[10:])}
    for i, j, k in itertools.product(range(3), repeat=3):
        c = [0, 0, 0]
        for a in (i, j, k):
            c[a] += 1
        Q = mono3[tuple(c)] - (u[i] * P[j, k] + u[j] * P[i, k] + u[k] * P[i, j]) + 2 * n * u[i] * u[j] * u[k]
        central = np.sum(V[i] * V[j] * V[k] * f[0]) * dv3
        assert abs(Q - central) < 1e-12 * max(1, abs(central))


def discrete_moments(sp, theta, orc):
    M = orc.maxwellian_grid(theta, orc_species(orc, sp), 3)
    v = [sp.vcentres(k) for k in range(3)]
    VZ, VY, VX = np.meshgrid(v[2], v[1], v[0], indexing="ij")
    V = [VX.ravel(), VY.ravel(), VZ.ravel()]
    dv3 = np.prod(sp.dv)
    out = [M.sum() * dv3]
    out += [np.sum(M * V[a]) * dv3 for a in range(3)]
    out += [np.sum(M * V[a] * V[b]) * dv3 for a, b in ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))]
    return np.array(out)


def targets_from(n, u, Th):
    E2 = n * (Th + np.outer(u, u))
    return np.array([n, n * u[0], n * u[1], n * u[2], E2[0, 0], E2[0, 1], E2[0, 2], E2[1, 1], E2[1, 2],
                     E2[2, 2]])


@pytest.mark.parametrize("seed", range(10))
def test_fit_reproduces_targets_on_coarse_grid(orc, seed):
    rng = np.random.default_rng(seed)
    sp = box(12, 5.0)
    dv = sp.dv[0]
    n = rng.uniform(0.2, 2.0)
    u = rng.uniform(-1.5, 1.5, 3)
    A = rng.normal(0, 0.25, (3, 3))
    Th = (np.diag(rng.uniform(0.6, 2.5, 3)) + A @ A.T) * dv ** 2
    T = targets_from(n, u, Th)
    theta, it, st = orc.maxent_fit(T, orc_species(orc, sp), 3, 1e-13, 30)
    assert st == 0
    D = discrete_moments(sp, theta, orc)
    scale = np.array([n] + [n * dv] * 3 + [n * dv * dv] * 6)
    assert np.max(np.abs(D - T) / scale) < 1e-11


def test_fit_tends_to_targets_on_fine_grid(orc):
    sp = box(40, 8.0)
    n, u = 0.7, np.array([0.3, -0.6, 0.1])
    Th = np.array([[1.1, 0.1, 0.0], [0.1, 0.9, -0.2], [0.0, -0.2, 1.4]])
    theta, it, st = orc.maxent_fit(targets_from(n, u, Th), orc_species(orc, sp), 3, 1e-13, 30)
    assert st == 0
    assert abs(theta[0] - n) < 1e-10
    np.testing.assert_allclose(theta[1:4], u, atol=1e-10)
    np.testing.assert_allclose(theta[[4, 5, 6, 7, 8, 9]], Th[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]], atol=1e-10)


def test_fit_1d_agrees_with_scipy_root(orc):
    from scipy.optimize import fsolve
    sp = W.SpeciesCfg("e", -1.0, 1.0, (10, 1, 1), (-3.0, 0, 0), (3.0, 1, 1))
    v = sp.vcentres(0)
    dv = sp.dv[0]
    n, u, th = 1.1, 0.37, 0.45 * dv * dv * 4
    T = np.array([n, n * u, n * (th + u * u)])
    theta, it, st = orc.maxent_fit(T, orc_species(orc, sp), 1, 1e-14, 40)
    assert st == 0

    def resid(p):
        nn, uu, tt = p[0], p[1], abs(p[2])
        M = nn / math.sqrt(2 * math.pi * tt) * np.exp(-(v - uu) ** 2 / (2 * tt))
        return [M.sum() * dv - T[0], (M * v).sum() * dv - T[1], (M * v * v).sum() * dv - T[2]]

    root = fsolve(resid, [n * 1.05, u + 0.1, th * 0.8], xtol=1e-13)
    np.testing.assert_allclose(theta, [root[0], root[1], abs(root[2])], rtol=1e-9, atol=1e-12)


def test_fit_3d_is_unique_scipy_from_other_starts(orc):
    """The discrete ten-moment fit (Sec. 2.2; c4) has one solution: scipy's
    hybrid root finder on a plain numpy evaluation of the discrete moments of
    M_theta (its own code path: an explicit sum over the cell centres),
    started from three different parameter sets, lands on the oracle's
    Newton solution, for a drifting, anisotropic, correlated Maxwellian on a
    coarse 8^3 grid where the discrete fit differs from the continuous
    Maxwellian at the 1e-2 level."""
    from scipy.optimize import root
    sp = box(8, 4.0)
    v = [sp.vcentres(a) for a in range(3)]
    VZ, VY, VX = np.meshgrid(v[2], v[1], v[0], indexing="ij")
    V = np.stack([VX, VY, VZ], -1).reshape(-1, 3)
    dv3 = float(np.prod(sp.dv))
    n, u = 1.3, np.array([0.3, -0.2, 0.1])
    Th = np.array([[0.9, 0.2, -0.1], [0.2, 0.7, 0.15], [-0.1, 0.15, 1.1]])
    T = targets_from(n, u, Th)
    th, it, st = orc.maxent_fit(T, orc_species(orc, sp), 3, 1e-13, 40)
    assert st == 0
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]

    def unpack(p):
        m = np.zeros((3, 3))
        for k, (a, b) in enumerate(pairs):
            m[a, b] = m[b, a] = p[4 + k]
        return p[0], p[1:4], m

    def resid(p):
        nn, uu, tt = unpack(p)
        w = V - uu
        q = np.einsum("ia,ab,ib->i", w, np.linalg.inv(tt), w)
        M = nn * np.exp(-0.5 * q) / math.sqrt((2 * math.pi) ** 3 * np.linalg.det(tt)) * dv3
        E2 = np.einsum("i,ia,ib->ab", M, V, V)
        return np.concatenate([[M.sum()], M @ V, [E2[a, b] for a, b in pairs]]) - T

    cont = np.concatenate([[n], u, [Th[a, b] for a, b in pairs]])
    assert np.abs(th - cont).max() > 1e-3  # the discrete fit is not the continuous Maxwellian
    for scale in (0.9, 1.1, 1.25):
        start = cont.copy()
        start[0] *= scale
        start[1:4] += 0.1 * (scale - 1.0)
        start[4:] *= scale
        sol = root(resid, start, method="hybr", tol=1e-12)
        assert np.abs(resid(sol.x)).max() < 1e-12 * n, sol.message
        np.testing.assert_allclose(sol.x, th, rtol=1e-8, atol=1e-11)


def test_fit_infeasible_falls_back(orc):
    """A variance below what any grid function with that mean can have (mean
    half-way between two cell centres, Theta << dv^2) cannot be fitted: the
    oracle reports the fallback and returns the continuous Maxwellian."""
    sp = box(10, 5.0)
    dv = sp.dv[0]
    n, u = 1.0, np.array([0.5 * dv, 0.0, 0.0])  # mid-way between centres
    Th = np.diag([0.01 * dv * dv, 1.0, 1.0])
    theta, it, st = orc.maxent_fit(targets_from(n, u, Th), orc_species(orc, sp), 3, 1e-12, 20)
    assert st == 1
    np.testing.assert_allclose(theta[:4], [n, u[0], 0, 0], atol=1e-15)
    theta, it, st = orc.maxent_fit(np.array([-1.0] + [0] * 9), orc_species(orc, sp), 3, 1e-12, 20)
    assert st == 2 and theta[0] == 0.0


def _fit_setup(orc, nv=10, ncell=4, seed=0):
    sp = box(nv, 4.0, q=-1.0, m=0.04)
    g = orc.make_grid(3, ncell, 1, 0.0, 1.0, 0.0, 1.0, 0)
    return sp, g


def test_exchange_recovers_fluid_moments(orc):
    sp, g = _fit_setup(orc)
    s = orc_species(orc, sp)
    rng = np.random.default_rng(21)
    dv = sp.dv[0]
    fs, fluid = [], []
    for c in range(4):
        n, u = rng.uniform(0.5, 1.5), rng.uniform(-0.5, 0.5, 3)
        Th = np.diag(rng.uniform(1.5, 3.0, 3)) * dv * dv
        base = sampled_maxwellian(sp, n, u, Th).ravel()
        pert = 1.0 + 0.05 * rng.uniform(-1, 1, base.size)  # non-Maxwellian part
        fs.append(base * pert)
        # fluid: slightly different u, T, and a density that differs by 1%
        fluid.append(targets_from(n * 1.01, u + 0.02 * dv, Th * 1.03))
    f = np.ascontiguousarray(np.stack(fs))
    U = np.ascontiguousarray(np.stack(fluid))
    nV = orc.moments(f, g, s)[:, 0].copy()
    stats = orc.moment_fit(f, g, s, U, 1e-13, 30)
    assert stats[1] == 0 and stats[2] == 0  # no fallback, no clipping
    mom = orc.moments(f, g, s)
    np.testing.assert_allclose(mom[:, 0], nV, rtol=1e-13)
    np.testing.assert_allclose(U[:, 0], nV, rtol=1e-14)  # fluid rescaled to n_V
    for c in range(4):
        scale = np.array([nV[c]] + [nV[c] * dv] * 3 + [nV[c] * dv * dv] * 6)
        assert np.max(np.abs(mom[c, :10] - U[c]) / scale) < 1e-10
    assert f.min() >= 0.0


def test_exchange_clips_and_keeps_density(orc):
    sp, g = _fit_setup(orc, ncell=3)
    s = orc_species(orc, sp)
    dv = sp.dv[0]
    f = np.ascontiguousarray(np.stack([sampled_maxwellian(sp, 1.0, np.zeros(3), np.eye(3) * 2 * dv * dv).ravel()
                                       for _ in range(3)]))
    f[:, ::7] *= 0.2  # holes where the exchange will go negative
    U = np.ascontiguousarray(np.stack([targets_from(1.0, np.array([1.5 * dv, 0, 0]), np.eye(3) * 1.2 * dv * dv)
                                       for _ in range(3)]))
    nV = orc.moments(f, g, s)[:, 0].copy()
    stats = orc.moment_fit(f, g, s, U, 1e-12, 30)
    assert stats[2] == 3  # every cell clipped
    assert f.min() >= 0.0
    np.testing.assert_allclose(orc.moments(f, g, s)[:, 0], nV, rtol=1e-14)


def test_exchange_leaves_maxwellian_unchanged(orc):
    sp, g = _fit_setup(orc, ncell=2)
    s = orc_species(orc, sp)
    dv = sp.dv[0]
    theta = np.array([0.9, 0.3 * dv, -0.2 * dv, 0.1 * dv, 2.0 * dv * dv, 0.1 * dv * dv, 0.0, 1.7 * dv * dv, 0.0,
                      2.2 * dv * dv])
    M = orc.maxwellian_grid(theta, s, 3)
    f = np.ascontiguousarray(np.stack([M, M]))
    U = np.ascontiguousarray(orc.moments(f, g, s)[:, :10].copy())
    f0 = f.copy()
    orc.moment_fit(f, g, s, U, 1e-13, 30)
    np.testing.assert_allclose(f, f0, rtol=0, atol=1e-12 * f0.max())
