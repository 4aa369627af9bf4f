"""Pins of the oracle's ten-moment fluid step (paper Sec. 2.1 equations, CWENO
of Kurganov-Levy 2000 with SSP-RK3 of Shu-Osher 1988) and field solvers (FDTD
of Sec. 2.1, Poisson of Sec. 3.1).

What fixes them:
* density is conserved to rounding (periodic and walls);
* with Q = 0 and no fields the system is linear with a closed-form solution
  (n quadratic in t, nu linear, E2 constant), reached at third order in dx;
* a uniform plasma in B_z gyrates: nu rotates at the cyclotron frequency;
* the Yee leapfrog reproduces the discrete dispersion relation exactly for a
  single Fourier mode (cos(omega h) = 1 - (c kappa h)^2 / 2), and a uniform
  current drives E by -c^2 J t;
* Poisson: E = sin(k x)/k for rho = cos(k x), at second order.
"""
import math

import numpy as np
import pytest

from paper_2109_06743_gb300 import workloads as W


def sp3(orc, q=1.0, m=1.0):
    return orc.make_species(q, m, (4, 4, 4), (-1, -1, -1), (1, 1, 1))


def test_fluid_conserves_density_periodic_and_walls(orc):
    for bc in (0, 1):
        nx, ny = 8, 6
        g = orc.make_grid(3, nx, ny, 0.0, 0.5, 0.0, 0.5, bc)
        rng = np.random.default_rng(bc)
        n = 1.0 + 0.2 * rng.uniform(size=(ny * nx))
        u = 0.1 * rng.normal(size=(ny * nx, 3))
        U = np.zeros((ny * nx, 10))
        U[:, 0] = n
        U[:, 1:4] = n[:, None] * u
        for k, (a, b) in enumerate(((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))):
            U[:, 4 + k] = n * (u[:, a] * u[:, b] + (0.5 if a == b else 0.0))
        Q = 0.01 * rng.normal(size=(ny * nx, 10))
        EB = W.random_fields(ny * nx, 3, 0.1, 0.5)
        m0 = U[:, 0].sum()
        orc.fluid_step(U, g, sp3(orc), Q, Q, Q, EB, 0.02)
        assert abs(U[:, 0].sum() - m0) < 1e-14 * m0


def test_fluid_linear_solution_third_order(orc):
    """Q = 0, E = B = 0, data varying in x only: n(t) = n0 - t d(nu0)/dx +
    t^2/2 d2(E2xx)/dx2, nu_x(t) = nu0 - t d(E2xx)/dx, E2 constant. Cell averages
    of the closed form are compared after t = 0.05 (L1 norm, dt ~ dx; the
    CWENO weights reach their linear values on these grids)."""
    errs = []
    for nx in (128, 256, 512):
        L = 1.0
        dx = L / nx
        g = orc.make_grid(3, nx, 1, 0.0, dx, 0.0, 1.0, 0)
        x = np.arange(nx + 1) * dx
        k = 2 * math.pi

        def avg(prim):
            return (prim(x[1:]) - prim(x[:-1])) / dx
        # n0 = 2 + 0.3 sin(kx), nu0 = 0.2 cos(kx), E2xx = 3 + 0.1 sin(kx)
        U = np.zeros((nx, 10))
        U[:, 0] = avg(lambda s: 2 * s - 0.3 * np.cos(k * s) / k)
        U[:, 1] = avg(lambda s: 0.2 * np.sin(k * s) / k)
        U[:, 4] = avg(lambda s: 3 * s - 0.1 * np.cos(k * s) / k)
        U[:, 7] = 1.0
        U[:, 9] = 1.0
        Q = np.zeros((nx, 10))
        EB = np.zeros((nx, 6))
        t = 0.05
        nsteps = nx // 4
        for _ in range(nsteps):
            orc.fluid_step(U, g, sp3(orc), Q, Q, Q, EB, t / nsteps)
        # closed form
        n_ex = avg(lambda s: 2 * s - 0.3 * np.cos(k * s) / k
                   - t * 0.2 * np.cos(k * s)          # -t d(nu0)/dx integrated: -t * nu0
                   + 0.5 * t * t * 0.1 * k * np.cos(k * s))  # t^2/2 d(E2)/dx integrated
        nu_ex = avg(lambda s: 0.2 * np.sin(k * s) / k - t * 0.1 * np.sin(k * s))
        errs.append(np.abs(U[:, 0] - n_ex).mean() + np.abs(U[:, 1] - nu_ex).mean())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 2.5, (errs, orders)


def test_fluid_gyration(orc):
    g = orc.make_grid(3, 2, 2, 0.0, 1.0, 0.0, 1.0, 0)
    U = np.zeros((4, 10))
    U[:, 0] = 1.0
    U[:, 1] = 1.0  # u = (1, 0, 0)
    U[:, 4] = 1.0 + 0.5
    U[:, 7] = 0.5
    U[:, 9] = 0.5
    EB = np.zeros((4, 6))
    EB[:, 5] = 2.0
    qm = -3.0
    sp = orc.make_species(-3.0, 1.0, (4, 4, 4), (-1, -1, -1), (1, 1, 1))
    Q = np.zeros((4, 10))
    dt, nsteps = 0.01, 50
    for _ in range(nsteps):
        orc.fluid_step(U, g, sp, Q, Q, Q, EB, dt)
    # d(nu_x + i nu_y)/dt = -i qm B_z (nu_x + i nu_y): SSP-RK3 multiplies by
    # the cubic Taylor polynomial R(z) = 1 + z + z^2/2 + z^3/6 each step
    z = -1j * qm * 2.0 * dt
    w = (1 + z + z * z / 2 + z ** 3 / 6) ** nsteps
    np.testing.assert_allclose(U[0, 1:3], [w.real, w.imag], atol=1e-13)
    ang = -qm * 2.0 * dt * nsteps  # exact gyration angle, to RK3 accuracy
    np.testing.assert_allclose(U[0, 1:3], [math.cos(ang), math.sin(ang)], atol=1e-4)
    # E2 = n (Theta + u u) rotates with u; the trace is conserved
    np.testing.assert_allclose(U[0, 4] + U[0, 7] + U[0, 9], 2.5, atol=1e-9)


def test_fluid_acceleration_by_a_uniform_e_field_is_exact(orc):
    """Eqs. 2-4 with B = 0 and a uniform E on a uniform state: the fluxes
    vanish and the sources give d(nu)/dt = (q/m) n E and
    d(E2_ab)/dt = (q/m)(nu_a E_b + nu_b E_a), so nu is linear and E2 quadratic
    in t, which SSP-RK3 integrates exactly. One step equals the closed form
    n u + (q/m) n E t, E2 + (q/m)(nu E + E nu) t + (q/m)^2 n E E t^2 to
    rounding (pins the signs, the factor q/m and the symmetrisation of the
    E2 source); the work done, (m/2) d tr(E2), is q t E . (nu + (q/m) n E t/2)."""
    g = orc.make_grid(3, 3, 2, 0.0, 1.0, 0.0, 1.0, 0)
    n, u = 1.4, np.array([0.3, -0.5, 0.2])
    th = np.array([[0.6, 0.1, 0.0], [0.1, 0.5, -0.05], [0.0, -0.05, 0.7]])
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    U0 = np.array([n, *(n * u)] + [n * (th[a, b] + u[a] * u[b]) for a, b in pairs])
    U = np.tile(U0, (6, 1))
    E = np.array([0.7, -0.4, 1.1])
    EB = np.zeros((6, 6))
    EB[:, :3] = E
    q, m = -2.0, 0.5
    qm = q / m
    sp = orc.make_species(q, m, (4, 4, 4), (-1, -1, -1), (1, 1, 1))
    Q = np.zeros((6, 10))
    t = 0.03
    orc.fluid_step(U, g, sp, Q, Q, Q, EB, t)
    nu = n * u
    nu_t = nu + qm * n * E * t
    E2 = n * (th + np.outer(u, u))
    E2_t = E2 + qm * (np.outer(nu, E) + np.outer(E, nu)) * t + qm * qm * n * np.outer(E, E) * t * t
    want = np.array([n, *nu_t] + [E2_t[a, b] for a, b in pairs])
    for c in range(6):
        np.testing.assert_allclose(U[c], want, rtol=0, atol=1e-14)
    work = 0.5 * m * (np.trace(E2_t) - np.trace(E2))
    assert abs(work - q * t * E @ (nu + 0.5 * qm * n * E * t)) < 1e-14


def _mode_test(orc, nx, ny, comp_e, comp_b, along):
    c = 3.0
    g = orc.make_grid(3, nx, ny, 0.0, 0.25, 0.0, 0.25, 0)
    yee = np.zeros((6, ny + 1, nx))
    k = 2 * math.pi / (nx * 0.25 if along == 0 else ny * 0.25)
    h = 0.02
    if along == 0:
        xi = np.arange(nx) * 0.25
        yee[comp_e, :, :] = np.cos(k * xi)[None, :]
        kappa = 2 * math.sin(k * 0.25 / 2) / 0.25
    else:
        yj = np.arange(ny + 1) * 0.25
        yee[comp_e, :, :] = np.cos(k * yj)[:, None]
        kappa = 2 * math.sin(k * 0.25 / 2) / 0.25
    yee = np.ascontiguousarray(yee.reshape(-1))
    J = np.zeros((nx * ny, 3))
    nsteps = 37
    for _ in range(nsteps):
        orc.maxwell(yee, g, J, h, c)
    th = math.acos(1 - (c * kappa * h) ** 2 / 2)
    e = yee.reshape(6, ny + 1, nx)[comp_e]
    return e[0, 0], math.cos(nsteps * th)


def test_yee_discrete_dispersion(orc):
    # Ez with By, wave along x
    got, ref = _mode_test(orc, 16, 4, 2, 4, 0)
    assert abs(got - ref) < 1e-12
    # Ez with Bx, wave along y (periodic y)
    got, ref = _mode_test(orc, 4, 16, 2, 3, 1)
    assert abs(got - ref) < 1e-12


def test_yee_current_drive_sign(orc):
    g = orc.make_grid(3, 4, 4, 0.0, 1.0, 0.0, 1.0, 0)
    yee = np.zeros(6 * 5 * 4)
    J = np.zeros((16, 3))
    J[:, 0] = 0.3
    J[:, 2] = -0.2
    c, h = 2.0, 0.1
    for _ in range(5):
        orc.maxwell(yee, g, J, h, c)
    y = yee.reshape(6, 5, 4)
    np.testing.assert_allclose(y[0], -c * c * 0.3 * 0.5, rtol=1e-14)
    np.testing.assert_allclose(y[2], c * c * 0.2 * 0.5, rtol=1e-14)
    np.testing.assert_allclose(y[3:], 0.0, atol=1e-15)


def test_yee_walls_keep_tangential_e_zero_and_energy_bounded(orc):
    nx, ny = 8, 8
    g = orc.make_grid(3, nx, ny, 0.0, 0.5, 0.0, 0.5, 1)
    rng = np.random.default_rng(2)
    yee = rng.normal(size=(6, ny + 1, nx))
    yee[0, 0] = yee[0, ny] = 0.0
    yee[2, 0] = yee[2, ny] = 0.0
    yee[[1, 3, 5], ny] = 0.0
    yee = np.ascontiguousarray(yee.reshape(-1))
    c = 1.0

    def energy(y):
        y = y.reshape(6, ny + 1, nx)
        return (y[0] ** 2).sum() / c ** 2 + (y[1, :ny] ** 2).sum() / c ** 2 + (y[2] ** 2).sum() / c ** 2 + \
            (y[3, :ny] ** 2).sum() + (y[4] ** 2).sum() + (y[5, :ny] ** 2).sum()
    e0 = energy(yee)
    for _ in range(200):
        orc.maxwell(yee, g, np.zeros((nx * ny, 3)), 0.1, c)
    y = yee.reshape(6, ny + 1, nx)
    assert np.all(y[0, 0] == 0) and np.all(y[0, ny] == 0) and np.all(y[2, 0] == 0) and np.all(y[2, ny] == 0)
    assert abs(energy(yee) / e0 - 1) < 0.2  # leapfrog: bounded, no growth


def test_poisson_second_order(orc):
    errs = []
    for nx in (32, 64):
        L = 4 * math.pi
        dx = L / nx
        x = (np.arange(nx) + 0.5) * dx
        k = 0.5
        edges = np.arange(nx + 1) * dx
        rho = (np.sin(k * edges[1:]) - np.sin(k * edges[:-1])) / (k * dx)  # cell averages of cos(kx)
        E = orc.poisson_1d(rho, dx)
        errs.append(np.abs(E - np.sin(k * x) / k).max())
    assert errs[0] < 1.5e-2 and math.log2(errs[0] / errs[1]) > 1.9


def test_fields_to_centres_is_exact_for_linear_fields(orc):
    """Reading: each Yee component is averaged from its staggered points to
    the cell centre by the symmetric 2- or 4-point mean (Bz is already
    there). A field linear in its position, a + b x + c y, is then exact at
    every centre away from the periodic wrap in x."""
    nx, ny, x0, dx, y0, dy = 10, 7, -1.0, 0.3, -0.7, 0.2
    g = orc.make_grid(3, nx, ny, x0, dx, y0, dy, 1)
    xs_int, xs_half = x0 + np.arange(nx) * dx, x0 + (np.arange(nx) + 0.5) * dx
    ys_int, ys_half = y0 + np.arange(ny + 1) * dy, y0 + (np.arange(ny + 1) + 0.5) * dy
    # positions (x, y) of each plane's points: Ex(i+1/2, j), Ey(i, j+1/2),
    # Ez(i, j), Bx(i, j+1/2), By(i+1/2, j), Bz(i+1/2, j+1/2)
    pos = [(xs_half, ys_int), (xs_int, ys_half), (xs_int, ys_int), (xs_int, ys_half), (xs_half, ys_int),
           (xs_half, ys_half)]
    coef = [(0.3, 1.1, -0.7), (-0.2, 0.4, 0.9), (1.5, -0.6, 0.25), (0.05, 0.8, -1.2), (0.7, -0.3, 0.6),
            (-0.4, 0.2, 1.3)]
    yee = np.zeros((6, ny + 1, nx))
    for k, ((px, py), (a, b, c)) in enumerate(zip(pos, coef)):
        yee[k] = a + b * px[None, :] + c * py[:, None]
    EB = orc.fields_to_centres(np.ascontiguousarray(yee.reshape(-1)), g).reshape(ny, nx, 6)
    xc, yc = x0 + (np.arange(nx) + 0.5) * dx, y0 + (np.arange(ny) + 0.5) * dy
    for k, (a, b, c) in enumerate(coef):
        want = a + b * xc[None, :] + c * yc[:, None]
        np.testing.assert_allclose(EB[:, 1:nx - 1, k], want[:, 1:nx - 1], rtol=0, atol=1e-13, err_msg=str(k))
