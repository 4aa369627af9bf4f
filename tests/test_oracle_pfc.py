"""Pins of the oracle's PFC scheme (Filbet, Sonnendruecker, Bertrand 2001, the
advection scheme of paper Sec. 2.1) against what the scheme's definition and
the paper fix: mass and flux conservation, positivity (Sec. 1, Sec. 2.1),
exact integer shifts, exactness for quadratic profiles (the reconstruction is
the cubic interpolant of the primitive), third-order convergence, and a brute
force integral of the interpolated primitive on tiny lines."""
import math

import numpy as np
import pytest

from paper_2109_06743_gb300 import workloads as W


def periodic_ext(f, ng):
    return np.concatenate([f[-ng:], f, f[:ng]])


def zero_ext(f, ng):
    return np.concatenate([np.zeros(ng), f, np.zeros(ng)])


@pytest.mark.parametrize("c", [0.0, 0.3, -0.3, 0.999, -0.999, 1.0, 1.7, -2.4, 3.25, -3.75])
def test_mass_periodic(orc, c):
    f = W.random_blocks(37, 1) + 0.01
    ng = int(math.floor(abs(c))) + 3
    out = orc.pfc_line(periodic_ext(f, ng), 37, ng, c)
    assert abs(out.sum() - f.sum()) <= 1e-14 * f.sum()


@pytest.mark.parametrize("c", [0.3, -0.3, 1.7, -2.4, 3.25, -3.75])
def test_mass_zero_flux(orc, c):
    f = W.random_blocks(23, 2) + 0.01
    ng = int(math.floor(abs(c))) + 3
    out = orc.pfc_line(zero_ext(f, ng), 23, ng, c, zero_flux=True)
    assert abs(out.sum() - f.sum()) <= 1e-14 * f.sum()
    assert out.min() >= 0.0


def test_positivity_random(orc):
    rng = np.random.default_rng(3)
    for trial in range(400):
        n = int(rng.integers(4, 40))
        f = rng.uniform(0, 1, n) ** 6  # spiky, many near-zero values
        f[rng.uniform(size=n) < 0.3] = 0.0
        c = rng.uniform(-4, 4)
        ng = int(math.floor(abs(c))) + 3
        zf = bool(trial % 2)
        ext = zero_ext(f, ng) if zf else periodic_ext(f, ng)
        if not zf and ng > n:
            continue
        out = orc.pfc_line(ext, n, ng, c, zero_flux=zf)
        assert out.min() >= -1e-15 * max(f.max(), 1e-300), (trial, c)


@pytest.mark.parametrize("s", [1, 2, -1, -3])
def test_integer_shift_is_exact(orc, s):
    f = W.random_blocks(19, 4)
    ng = abs(s) + 3
    out = orc.pfc_line(periodic_ext(f, ng), 19, ng, float(s))
    np.testing.assert_allclose(out, np.roll(f, s), rtol=0, atol=1e-15)


@pytest.mark.parametrize("c", [0.25, 0.8, -0.4, 1.6, -2.3])
def test_exact_for_quadratics(orc, c):
    """The PFC flux integrates the cubic interpolant of the primitive, so it
    is exact for quadratic f when the limiter is inactive (f large and
    smooth). The result must equal the exact cell averages of f(x - c dx)."""
    a, b, q = 5.0, 0.3, 0.02
    n, ng = 12, int(math.floor(abs(c))) + 3
    edges = np.arange(-ng, n + ng + 1, dtype=float)  # dx = 1

    def prim(x):
        return a * x + b * x ** 2 / 2 + q * x ** 3 / 3

    avg = (prim(edges[1:]) - prim(edges[:-1]))
    out = orc.pfc_line(avg, n, ng, c)
    e = edges[ng:ng + n + 1] - c
    exact = prim(e[1:]) - prim(e[:-1])
    np.testing.assert_allclose(out, exact, rtol=0, atol=1e-12)


def test_unlimited_flux_is_integral_of_interpolated_primitive(orc):
    """Brute force on tiny lines: for data where the limiter is inactive the
    flux through an interface equals the integral, over the part of the foot
    cell that crosses it, of the derivative of the cubic through the primitive
    at the four interfaces of cells j-1, j, j+1 (numpy.polyfit, an
    independent construction)."""
    rng = np.random.default_rng(5)
    for trial in range(50):
        n = 6
        f = 10.0 + rng.uniform(0, 1, n + 6)  # limiter inactive: |df| < 2 f
        alpha = rng.uniform(0.01, 0.99)
        ng = 3
        out = orc.pfc_line(f, n, ng, alpha)
        fc = f[ng:ng + n]
        # flux through interface i+1/2 for positive shift alpha (foot in cell i)
        phi = []
        for i in range(-1, n):
            j = i + ng
            xs = np.array([-1.0, 0.0, 1.0, 2.0])  # interfaces j-3/2 .. j+3/2 (cell j = [0,1])
            F = np.array([0.0, f[j - 1], f[j - 1] + f[j], f[j - 1] + f[j] + f[j + 1]])
            p = np.polyfit(xs, F, 3)
            phi.append(np.polyval(p, 1.0) - np.polyval(p, 1.0 - alpha))
        phi = np.array(phi)
        brute = fc + phi[:-1] - phi[1:]
        np.testing.assert_allclose(out, brute, rtol=1e-12, atol=1e-12)


def test_third_order_convergence(orc):
    """Smooth periodic data (limiter inactive) shifted by 0.37 cells per step
    for N steps: the error against exact cell averages falls ~ N^-3."""
    errs = []
    for n in (32, 64, 128):
        x = np.arange(n + 1) / n

        def prim(xx):
            return 2.0 * xx - np.cos(2 * math.pi * xx) / (2 * math.pi)

        f = (prim(x[1:]) - prim(x[:-1])) * n
        c = 0.37
        ng = 3
        g = f.copy()
        for _ in range(n):
            g = orc.pfc_line(periodic_ext(g, ng), n, ng, c)
        shift = c  # domain fraction after n steps of c cells
        exact = (prim(x[1:] - shift) - prim(x[:-1] - shift)) * n
        errs.append(np.abs(g - exact).max())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(orders) > 2.7, (errs, orders)


def test_space_sweep_wall_conserves_mass_and_mirror_symmetry(orc):
    """y sweep with reflecting walls (Sec. 3.3): ghosts f(-y, v_y) = f(y, -v_y)
    conserve the total mass, and data symmetric under (y, v_y) -> (-y, -v_y)
    stays symmetric."""
    cfg = W.harris(nx=3, ny=10, nv=6, steps=1)
    sp = cfg.species[0]
    g = orc.make_grid(3, cfg.nx, cfg.ny, cfg.x0, cfg.dx, cfg.y0, cfg.dy, 1)
    s = orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)
    f = W.random_blocks((cfg.ny, cfg.nx, 6, 6, 6), 7)
    f = 0.5 * (f + f[::-1, :, :, ::-1, :])  # symmetric under y -> -y, v_y -> -v_y
    f = np.ascontiguousarray(f.reshape(cfg.ncell, -1))
    m0 = f.sum()
    dt = 1.7 * cfg.dy / abs(sp.vmin[1])  # CFL > 1 at the box edge
    orc.advect_space(f, g, s, 1, dt)
    assert abs(f.sum() - m0) <= 1e-14 * m0
    f5 = f.reshape(cfg.ny, cfg.nx, 6, 6, 6)
    np.testing.assert_allclose(f5, f5[::-1, :, :, ::-1, :], rtol=1e-13, atol=1e-15)
    assert f.min() >= 0.0


def test_space_sweep_x_matches_line_steps(orc):
    """The x sweep applies the periodic line step with c = v_x dt / dx to every
    (y, velocity) line."""
    cfg = W.harris(nx=9, ny=2, nv=4, steps=1)
    sp = cfg.species[1]
    g = orc.make_grid(3, cfg.nx, cfg.ny, cfg.x0, cfg.dx, cfg.y0, cfg.dy, 1)
    s = orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)
    f0 = W.random_blocks((cfg.ny, cfg.nx, 4, 4, 4), 8)
    f = np.ascontiguousarray(f0.reshape(cfg.ncell, -1)).copy()
    dt = 2.3 * cfg.dx / abs(sp.vmin[0])
    orc.advect_space(f, g, s, 0, dt)
    f = f.reshape(f0.shape)
    vx = sp.vcentres(0)
    for j in range(cfg.ny):
        for k in range(4):
            for jj in range(4):
                for i in range(4):
                    c = vx[i] * dt / cfg.dx
                    ng = int(math.floor(abs(c))) + 3
                    line = f0[j, :, k, jj, i]
                    ref = orc.pfc_line(periodic_ext(line, ng), cfg.nx, ng, c)
                    np.testing.assert_allclose(f[j, :, k, jj, i], ref, rtol=0, atol=1e-15)
