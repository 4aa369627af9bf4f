"""Pins of the oracle's stand-alone fluid model with the gradient heat-flux
closure (Sec. 2.3, Eq. "gradient closure"; test infrastructure).

* The model's third moment E3_kab = u_k E2_ab + u_a E2_kb + u_b E2_ka -
  2 n u_k u_a u_b equals the raw third moment of a drifting, anisotropic
  Maxwellian summed on a fine velocity grid by the oracle's moment routine
  (a different code path: a plain midpoint sum over the grid).
* The closure source, isolated as L(U; chi) - L(U; 0), equals
  chi_k0 n v_t times the closed-form five-point Laplacian of
  theta_yy = theta0 + eps cos(k x), -eps cos(k x) (2 - 2 cos(k dx)) / dx^2,
  with v_t = sqrt(tr(theta) / 3), and vanishes in the other components.
* chi_k0 = chi d_s with chi = 2 sqrt(2/pi) and d_s = sqrt(m_s) / |q_s|
  (unit reference density, mu0 = 1): 1.5958 d_s; electrons of mass 1/100
  have d_e = 0.1.
* Conservation: on a periodic grid without fields the flux part changes
  neither the total of n, nu nor of E2 (telescoping interface fluxes), and
  with uniform n and tr(theta) the closure source sums to zero.
* A uniform state is stationary.
"""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def o(orc):
    return orc


def state_from(n, u, th):
    """(n, nu_a, E2_ab) from density, drift and theta (E2 = n (theta + u u))."""
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    return np.array([n, n * u[0], n * u[1], n * u[2]] + [n * (th[a][b] + u[a] * u[b]) for a, b in pairs])


def test_chi_over_k0():
    import oracle
    assert abs(oracle.CHI - 1.5957691216057308) < 1e-15
    assert abs(oracle.closure_chi_k0(-1.0, 0.01) - 0.1 * oracle.CHI) < 1e-15
    assert abs(oracle.closure_chi_k0(1.0, 1.0) - oracle.CHI) < 1e-15


def test_closure_third_moment_is_that_of_a_maxwellian(o):
    n, u = 1.7, np.array([0.3, -0.45, 0.2])
    th = np.array([[0.8, 0.15, -0.1], [0.15, 0.5, 0.05], [-0.1, 0.05, 0.65]])
    nv, half = 56, 8.0
    g = o.make_grid(3, 1, 1, 0.0, 1.0, 0.0, 1.0, 0)
    lo = [u[a] - half for a in range(3)]
    hi = [u[a] + half for a in range(3)]
    sp = o.make_species(-1.0, 1.0, (nv, nv, nv), lo, hi)
    dv = [(hi[a] - lo[a]) / nv for a in range(3)]
    ax = [lo[a] + (np.arange(nv) + 0.5) * dv[a] - u[a] for a in range(3)]
    VZ, VY, VX = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    w = np.stack([VX, VY, VZ], -1)
    ti = np.linalg.inv(th)
    q = np.einsum("...a,ab,...b->...", w, ti, w)
    f = n * np.exp(-0.5 * q) / math.sqrt((2 * math.pi) ** 3 * np.linalg.det(th))
    m = o.moments(f.reshape(1, -1), g, sp)[0]
    assert abs(m[0] - n) < 1e-10 * n
    U = np.concatenate([m[:4], m[4:10]])
    e3 = o.maxwellian_e3(U)
    scale = np.abs(m[10:20]).max()
    assert np.abs(e3 - m[10:20]).max() < 1e-9 * scale, (e3, m[10:20])
    # the exact form from (n, u, theta) agrees too
    e3x = o.maxwellian_e3(state_from(n, u, th))
    assert np.abs(e3x - m[10:20]).max() < 1e-9 * scale


def periodic_grid(o, nx=24, ny=8, lx=6.0, ly=2.0):
    return o.make_grid(3, nx, ny, 0.0, lx / nx, 0.0, ly / ny, 0), nx, ny, lx / nx


def test_closure_source_closed_form(o):
    g, nx, ny, dx = periodic_grid(o)
    sp = o.make_species(-1.0, 0.04, (8, 8, 8), (-3,) * 3, (3,) * 3)
    k = 2 * math.pi * 2 / (nx * dx)
    eps, t0, tx, tz = 0.05, 0.4, 0.3, 0.2
    x = (np.arange(nx) + 0.5) * dx
    U = np.zeros((ny, nx, 10))
    for i in range(nx):
        th = np.diag([tx, t0 + eps * math.cos(k * x[i]), tz])
        U[:, i] = state_from(1.3, np.zeros(3), th)
    U = U.reshape(-1, 10)
    EB = np.zeros((nx * ny, 6))
    chi_k0 = 0.37
    d = o.fluid_rhs_closure(U, g, sp, EB, chi_k0) - o.fluid_rhs_closure(U, g, sp, EB, 0.0)
    d = d.reshape(ny, nx, 10)
    lap = -eps * np.cos(k * x) * (2 - 2 * math.cos(k * dx)) / dx ** 2
    vt = np.sqrt((tx + t0 + eps * np.cos(k * x) + tz) / 3)
    want = chi_k0 * 1.3 * vt * lap
    for j in range(ny):
        assert np.allclose(d[j, :, 7], want, rtol=1e-12, atol=1e-14)
    others = [0, 1, 2, 3, 4, 5, 6, 8, 9]
    assert np.abs(d[..., others]).max() < 1e-13


def test_flux_part_conserves_and_closure_sums_to_zero(o):
    g, nx, ny, dx = periodic_grid(o, 20, 12, 5.0, 3.0)
    sp = o.make_species(1.0, 1.0, (8, 8, 8), (-3,) * 3, (3,) * 3)
    X, Y = np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny)
    U = np.zeros((ny, nx, 10))
    for j in range(ny):
        for i in range(nx):
            ph = 2 * math.pi * np.array([X[j, i], Y[j, i]])
            n = 1 + 0.2 * math.sin(ph[0]) * math.cos(ph[1])
            u = 0.1 * np.array([math.cos(ph[1]), math.sin(ph[0]), math.sin(ph[0] + ph[1])])
            th = np.array([[0.5 + 0.1 * math.cos(ph[0]), 0.05, 0.0], [0.05, 0.4, 0.02 * math.sin(ph[1])],
                           [0.0, 0.02 * math.sin(ph[1]), 0.45]])
            U[j, i] = state_from(n, u, th)
    U = U.reshape(-1, 10)
    EB = np.zeros((nx * ny, 6))
    L0 = o.fluid_rhs_closure(U, g, sp, EB, 0.0)
    scale = np.abs(L0).max(axis=0) + 1e-300
    assert np.all(np.abs(L0.sum(axis=0)) <= 1e-12 * scale * nx * ny), L0.sum(axis=0) / scale
    # uniform n and tr(theta): n v_t is uniform and the closure source telescopes
    V = np.zeros((ny, nx, 10))
    for j in range(ny):
        for i in range(nx):
            ph = 2 * math.pi * np.array([X[j, i], Y[j, i]])
            a = 0.1 * math.sin(ph[0] + 2 * ph[1])
            V[j, i] = state_from(1.0, np.zeros(3), np.diag([0.5 + a, 0.5 - a, 0.5]))
    V = V.reshape(-1, 10)
    S = o.fluid_rhs_closure(V, g, sp, EB, 0.8) - o.fluid_rhs_closure(V, g, sp, EB, 0.0)
    assert np.abs(S).max() > 1e-3
    assert np.abs(S.sum(axis=0)).max() < 1e-12 * np.abs(S).max() * nx * ny


def test_uniform_state_is_stationary(o):
    g, nx, ny, dx = periodic_grid(o, 10, 6, 2.0, 1.2)
    sp = o.make_species(1.0, 1.0, (8, 8, 8), (-3,) * 3, (3,) * 3)
    U = np.tile(state_from(0.9, np.array([0.2, -0.1, 0.3]), np.diag([0.4, 0.5, 0.6]) + 0.05), (nx * ny, 1))
    EB = np.zeros((nx * ny, 6))
    L = o.fluid_rhs_closure(U, g, sp, EB, 0.5)
    assert np.abs(L).max() < 1e-13
    U1 = U.copy()
    o.fluid_step_closure(U1, g, sp, EB, 0.01, 0.5)
    assert np.abs(U1 - U).max() < 1e-13
