"""Pins of the oracle's velocity-space advection (paper Sec. 2.1: the Lorentz
term (q/m)(E + v x B).grad_v f with zero-flux velocity boundaries; the
velocity splitting is read as an exact factorisation of the Boris map into
five single-axis PFC shears).

What fixes it: the composed shears equal the Boris rotation written
independently with Rodrigues' formula (rotation by -2 atan(q|B|dt/2m) about
B) plus the two electric half kicks; density is conserved exactly; f stays
positive; B = 0 with whole-cell kicks is an exact shift; a drifting
Maxwellian's mean velocity rotates by the Boris angle."""
import math

import numpy as np
import pytest

from paper_2109_06743_gb300 import workloads as W


def rodrigues(axis, angle):
    a = np.asarray(axis, dtype=float)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) * math.cos(angle) + math.sin(angle) * K + (1 - math.cos(angle)) * np.outer(a, a)


def compose(sh):
    """Affine map (L, t) of the sweeps applied in order."""
    L, t = np.eye(3), np.zeros(3)
    for axis, c1, c2, c0 in sh:
        axis = int(axis)
        others = [b for b in range(3) if b != axis]
        S = np.eye(3)
        S[axis, others[0]] = c1
        S[axis, others[1]] = c2
        k = np.zeros(3)
        k[axis] = c0
        L, t = S @ L, S @ t + k
    return L, t


@pytest.mark.parametrize("seed", range(40))
def test_five_shears_compose_to_boris_map(orc, seed):
    rng = np.random.default_rng(seed)
    qm = rng.choice([-25.0, 1.0, -100.0])
    B = rng.normal(0, 1, 3)
    if seed % 4 == 1:
        B[rng.integers(3)] = 0.0  # field in a coordinate plane
    if seed % 4 == 2:
        B[:] = 0.0
        B[rng.integers(3)] = rng.normal()  # field along an axis
    E = rng.normal(0, 1, 3)
    dt = rng.uniform(0.001, 0.05)
    sh = orc.velocity_shears(qm, E, B, dt, 5)
    p = int(np.argmax(np.abs(B)))
    rest = [a for a in range(3) if a != p]
    assert [int(a) for a in sh[:, 0]] == [p, rest[0], rest[1], rest[0], p]
    L, t = compose(sh)
    theta = -2.0 * math.atan(abs(qm) * np.linalg.norm(B) * dt / 2.0) * np.sign(qm)
    R = rodrigues(B, theta) if np.linalg.norm(B) > 0 else np.eye(3)
    np.testing.assert_allclose(L, R, rtol=0, atol=1e-12)
    h = 0.5 * qm * dt * E
    np.testing.assert_allclose(t, R @ h + h, rtol=0, atol=1e-12)
    assert abs(np.linalg.det(L) - 1.0) < 1e-12
    if abs(theta) < 1.0:
        assert np.abs(sh[:, 1:3]).max() < 2.0  # shears stay bounded for moderate angles


def test_zero_field_gives_identity_shears(orc):
    sh = orc.velocity_shears(-25.0, np.zeros(3), np.zeros(3), 0.01, 5)
    assert np.all(sh[:, 1:] == 0.0)


def test_three_shear_split_is_the_lorentz_acceleration(orc):
    qm, dt = -25.0, 0.01
    E = np.array([0.1, -0.2, 0.3])
    B = np.array([0.5, 0.7, -1.1])
    sh = orc.velocity_shears(qm, E, B, dt, 3)
    v = np.array([0.3, -0.8, 1.2])
    for axis, c1, c2, c0 in sh:
        axis = int(axis)
        others = [b for b in range(3) if b != axis]
        acc = qm * (E + np.cross(v, B))[axis] * dt
        assert abs(c1 * v[others[0]] + c2 * v[others[1]] + c0 - acc) < 1e-14


@pytest.mark.parametrize("nshear", [5, 3])
def test_velocity_push_conserves_density_and_positivity(orc, nshear):
    cfg = W.harris(nx=3, ny=2, nv=8, steps=1)
    sp = cfg.species[0]
    g = orc.make_grid(3, cfg.nx, cfg.ny, cfg.x0, cfg.dx, cfg.y0, cfg.dy, 1)
    s = orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)
    f = W.random_blocks((cfg.ncell, 512), 11) ** 4
    m0 = f.sum(axis=1)
    EB = W.random_fields(cfg.ncell, 12, e_scale=2.0, b_scale=1.5)
    dt = 0.02
    orc.advect_velocity(f, g, s, EB, dt, nshear)
    np.testing.assert_allclose(f.sum(axis=1), m0, rtol=1e-14)
    assert f.min() >= -1e-15 * f.max()  # positive up to rounding


def test_velocity_push_whole_cell_kick_is_exact_shift(orc):
    """B = 0 and E chosen so that each component moves an integer number of
    cells: a blob away from the box edges is shifted exactly."""
    cfg = W.harris(nx=1, ny=1, nv=10, steps=1)
    sp = cfg.species[1]
    g = orc.make_grid(3, 1, 1, cfg.x0, cfg.dx, cfg.y0, cfg.dy, 1)
    s = orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)
    blob = np.zeros((10, 10, 10))
    blob[3:6, 2:5, 4:7] = W.random_blocks((3, 3, 3), 13) + 0.1
    shift = np.array([2, -1, 1])  # cells in x, y, z
    dt = 0.1
    E = shift * np.array(sp.dv) / (sp.q / sp.m * dt)
    EB = np.concatenate([E, np.zeros(3)])[None, :]
    f = np.ascontiguousarray(blob.reshape(1, -1)).copy()
    orc.advect_velocity(f, g, s, EB, dt, 5)
    ref = np.roll(np.roll(np.roll(blob, shift[0], axis=2), shift[1], axis=1), shift[2], axis=0)
    np.testing.assert_allclose(f.reshape(10, 10, 10), ref, rtol=0, atol=1e-14)


def test_drifting_maxwellian_rotates_by_boris_angle(orc):
    """E = 0, B along z: the mean velocity of a well-resolved drifting
    Maxwellian rotates by the Boris angle (closed form), its density and
    |u| are unchanged."""
    nv, vm = 24, 6.0
    sp = W.SpeciesCfg("i", 1.0, 1.0, (nv, nv, nv), (-vm,) * 3, (vm,) * 3)
    g = orc.make_grid(3, 1, 1, 0.0, 1.0, 0.0, 1.0, 0)
    s = orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)
    u0 = np.array([0.8, 0.3, -0.2])
    v = [sp.vcentres(a) for a in range(3)]
    VZ, VY, VX = np.meshgrid(v[2], v[1], v[0], indexing="ij")
    th = 0.6
    f = np.exp(-((VX - u0[0]) ** 2 + (VY - u0[1]) ** 2 + (VZ - u0[2]) ** 2) / (2 * th))
    f = np.ascontiguousarray(f.reshape(1, -1))
    Bz, dt = 2.0, 0.05
    EB = np.array([[0, 0, 0, 0, 0, Bz]], dtype=float)
    m0 = orc.moments(f, g, s)[0]
    orc.advect_velocity(f, g, s, EB, dt, 5)
    m1 = orc.moments(f, g, s)[0]
    assert abs(m1[0] - m0[0]) <= 1e-14 * m0[0]
    u1 = m1[1:4] / m1[0]
    ang = -2 * math.atan(Bz * dt / 2)
    R = rodrigues([0, 0, 1], ang)
    np.testing.assert_allclose(u1, R @ u0, atol=2e-3)
    assert abs(np.linalg.norm(u1) - np.linalg.norm(u0)) < 2e-3


def test_maxwellian_at_rest_is_invariant_under_b_and_drifts_with_e_cross_b(orc):
    """c2's physics pins of the velocity map. (1) E = 0, B along z: an
    isotropic Maxwellian at rest is invariant up to the scheme's
    discretisation error: density exact, mean velocity 0 to 1e-12 (mirror
    symmetries of the shears), and the numerical heating over ten steps
    vanishes as the grid is refined (measured 11%, 0.5%, 1e-4 at 16^3, 32^3,
    48^3 with the thermal speed 0.77 on +-6). (2) E = E_y y, B = B_z z: over
    whole gyration periods the mean velocity averages to the E x B drift
    E_y / B_z along x (Boris map: the drift is exact and the velocity
    rotates about it)."""
    vm, th = 6.0, 0.6
    g = orc.make_grid(3, 1, 1, 0.0, 1.0, 0.0, 1.0, 0)
    heat = {}
    for nv in (16, 32, 48):
        sp = W.SpeciesCfg("i", 1.0, 1.0, (nv, nv, nv), (-vm,) * 3, (vm,) * 3)
        s = orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)
        v = [sp.vcentres(a) for a in range(3)]
        VZ, VY, VX = np.meshgrid(v[2], v[1], v[0], indexing="ij")
        f = np.ascontiguousarray(np.exp(-(VX ** 2 + VY ** 2 + VZ ** 2) / (2 * th)).reshape(1, -1))
        m0 = orc.moments(f, g, s)[0]
        EB = np.array([[0, 0, 0, 0, 0, 2.0]], dtype=float)
        for _ in range(10):
            orc.advect_velocity(f, g, s, EB, 0.05, 5)
        m1 = orc.moments(f, g, s)[0]
        assert abs(m1[0] - m0[0]) <= 1e-13 * m0[0]
        assert np.abs(m1[1:4] / m1[0]).max() < 1e-12
        heat[nv] = (m1[4] + m1[7] + m1[9]) / m1[0] / ((m0[4] + m0[7] + m0[9]) / m0[0]) - 1.0
    assert 0 < heat[48] < 1e-3 and heat[48] < heat[32] / 10 < heat[16] / 100, heat
    nv = 24
    sp = W.SpeciesCfg("i", 1.0, 1.0, (nv, nv, nv), (-vm,) * 3, (vm,) * 3)
    s = orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)
    v = [sp.vcentres(a) for a in range(3)]
    VZ, VY, VX = np.meshgrid(v[2], v[1], v[0], indexing="ij")
    # E x B: Ey = 0.5, Bz = 2 -> drift 0.25 along x; the Boris rotation
    # angle per step is 2 atan(Bz dt / 2), so 40 steps of dt = 0.0785...
    # make whole periods
    f = np.ascontiguousarray(np.exp(-(VX ** 2 + VY ** 2 + VZ ** 2) / (2 * th)).reshape(1, -1))
    Ey, Bz = 0.5, 2.0
    nsteps = 40
    ang = 2 * math.pi / nsteps
    dt = 2 * math.tan(ang / 2) / Bz
    EB = np.array([[0, Ey, 0, 0, 0, Bz]], dtype=float)
    us = []
    for _ in range(nsteps):
        orc.advect_velocity(f, g, s, EB, dt, 5)
        m = orc.moments(f, g, s)[0]
        us.append(m[1:4] / m[0])
    ubar = np.mean(us, axis=0)
    assert abs(ubar[0] - Ey / Bz) < 5e-3, ubar
    assert abs(ubar[1]) < 5e-3 and abs(ubar[2]) < 1e-12, ubar


def test_velocity_push_1d(orc):
    """1D1V: one zero-flux sweep with c = (q/m) E dt / dv."""
    cfg = W.landau(nx=4, nv=16)
    sp = cfg.species[0]
    g = orc.make_grid(1, 4, 1, cfg.x0, cfg.dx)
    s = orc.make_species(sp.q, sp.m, sp.nv, sp.vmin, sp.vmax)
    f0 = W.random_blocks((4, 16), 17)
    f = f0.copy()
    EB = np.zeros((4, 6))
    EB[:, 0] = [0.5, -1.3, 2.2, 0.0]
    dt = 0.7
    orc.advect_velocity(f, g, s, EB, dt, 5)
    for c in range(4):
        cc = sp.q / sp.m * EB[c, 0] * dt / sp.dv[0]
        ng = int(math.floor(abs(cc))) + 3
        ref = orc.pfc_line(np.concatenate([np.zeros(ng), f0[c], np.zeros(ng)]), 16, ng, cc, zero_flux=True)
        np.testing.assert_allclose(f[c], ref, rtol=0, atol=1e-15)
