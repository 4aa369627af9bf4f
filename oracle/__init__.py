"""Plain FP64 CPU oracle of the moment-fitting PFC Vlasov solver (arXiv:2109.06743).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code with
the CUDA path (``paper_2109_06743_gb300``) and neither imports the other.

The C sources (``oracle/*.c``) follow the paper's definitions with plain loops;
this module compiles them with gcc into ``oracle/_build/liboracle.so`` and wraps
them with ctypes over numpy float64 arrays. Every routine's docstring names the
passage of the paper it follows.

Parity pins (tests/test_oracle_*.py) check it against what the paper and the
mathematics fix; see the module docstrings there.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["pfc.c", "moments.c", "maxent.c", "fluid.c", "fields.c"]
_LIB = None
_LOCK = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (host code only, portable C99)."""
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "liboracle.so")
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(so):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr, __file__])
        if os.path.getmtime(so) >= newest:
            return so
    tmp = so + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


class Grid(ctypes.Structure):
    _fields_ = [
        ("nvdim", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("x0", ctypes.c_double),
        ("dx", ctypes.c_double),
        ("y0", ctypes.c_double),
        ("dy", ctypes.c_double),
        ("bc_y", ctypes.c_int),
    ]


class Species(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_double),
        ("m", ctypes.c_double),
        ("nv", ctypes.c_int * 3),
        ("vmin", ctypes.c_double * 3),
        ("dv", ctypes.c_double * 3),
    ]


def make_grid(nvdim, nx, ny, x0, dx, y0=0.0, dy=1.0, bc_y=0) -> Grid:
    return Grid(nvdim, nx, ny, x0, dx, y0, dy, bc_y)


def make_species(q, m, nv, vmin, vmax) -> Species:
    nv = list(nv) + [1] * (3 - len(nv))
    vmin = list(vmin) + [0.0] * (3 - len(vmin))
    vmax = list(vmax) + [1.0] * (3 - len(vmax))
    dv = [(vmax[a] - vmin[a]) / nv[a] for a in range(3)]
    return Species(q, m, (ctypes.c_int * 3)(*nv), (ctypes.c_double * 3)(*vmin),
                   (ctypes.c_double * 3)(*dv))


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(build())
            G, S = ctypes.POINTER(Grid), ctypes.POINTER(Species)
            L.or_pfc_line.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp]
            L.or_advect_space.argtypes = [_dp, G, S, ctypes.c_int, ctypes.c_double]
            L.or_advect_velocity.argtypes = [_dp, G, S, _dp, ctypes.c_double, ctypes.c_int]
            L.or_velocity_shears.argtypes = [ctypes.c_double, _dp, _dp, ctypes.c_double, ctypes.c_int, _dp]
            L.or_moments.argtypes = [_dp, G, S, _dp]
            L.or_moments.restype = None
            L.or_maxent_fit.argtypes = [_dp, S, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _ip, _ip]
            L.or_maxwellian_grid.argtypes = [_dp, S, ctypes.c_int, _dp]
            L.or_maxwellian_grid.restype = None
            L.or_moment_fit.argtypes = [_dp, G, S, _dp, ctypes.c_double, ctypes.c_int, _lp]
            L.or_fluid_step.argtypes = [_dp, G, S, _dp, _dp, _dp, _dp, ctypes.c_double]
            L.or_fluid_step_closure.argtypes = [_dp, G, S, _dp, ctypes.c_double, ctypes.c_double]
            L.or_fluid_rhs_closure.argtypes = [_dp, G, S, _dp, ctypes.c_double, _dp]
            L.or_maxwellian_e3.argtypes = [_dp, _dp]
            L.or_maxwellian_e3.restype = None
            L.or_maxwell.argtypes = [_dp, G, _dp, ctypes.c_double, ctypes.c_double]
            L.or_fields_to_centres.argtypes = [_dp, G, _dp]
            L.or_fields_to_centres.restype = None
            L.or_poisson_1d.argtypes = [_dp, ctypes.c_int, ctypes.c_double, _dp]
            L.or_poisson_1d.restype = None
            _LIB = L
    return _LIB


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def pfc_line(fext, n, ng, c, zero_flux=False):
    """One conservative PFC step on an extended 1D line (Filbet et al. 2001,
    cited in Sec. 2.1). ``fext`` has ``ng`` ghosts on each side."""
    fext = np.ascontiguousarray(fext, dtype=np.float64)
    out = np.zeros(n)
    _check(lib().or_pfc_line(_d(fext), n, ng, float(c), int(bool(zero_flux)), _d(out)), "pfc_line")
    return out


def advect_space(f, grid, sp, axis, dt):
    """In-place spatial PFC sweep (Sec. 2.1; walls in y per Sec. 3.3)."""
    _check(lib().or_advect_space(_d(f), ctypes.byref(grid), ctypes.byref(sp), axis, dt), "advect_space")


def advect_velocity(f, grid, sp, EB, dt, nshear=5):
    """In-place velocity-space advection under (q/m)(E + v x B) (Sec. 2.1)."""
    EB = np.ascontiguousarray(EB, dtype=np.float64)
    _check(lib().or_advect_velocity(_d(f), ctypes.byref(grid), ctypes.byref(sp), _d(EB), dt, nshear),
           "advect_velocity")


def velocity_shears(qm, E, B, dt, nshear=5):
    """Shear factors of the Boris velocity map of one cell: [nshear, 4] =
    (axis, coefficient of the lower other axis, of the higher, constant)."""
    out = np.zeros(nshear * 4)
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    _check(lib().or_velocity_shears(qm, _d(E), _d(B), dt, nshear, _d(out)), "velocity_shears")
    return out.reshape(nshear, 4)


def moments(f, grid, sp):
    """Raw midpoint moments int v^alpha f dv (Sec. 2.1): [ncell, 20] or [ncell, 4]."""
    nm = 4 if grid.nvdim == 1 else 20
    out = np.zeros((grid.nx * grid.ny, nm))
    lib().or_moments(_d(np.ascontiguousarray(f)), ctypes.byref(grid), ctypes.byref(sp), _d(out))
    return out


def maxent_fit(target, sp, nvdim, tol=1e-12, max_iter=20):
    """Discrete ten-moment Maxwellian fit (Sec. 2.2 f_M; fitted so that its
    midpoint moments equal ``target``). Returns (theta, iters, status)."""
    target = np.ascontiguousarray(target, dtype=np.float64)
    theta = np.zeros(10)
    it = ctypes.c_int(0)
    st = ctypes.c_int(0)
    _check(lib().or_maxent_fit(_d(target), ctypes.byref(sp), nvdim, tol, max_iter, _d(theta),
                               ctypes.byref(it), ctypes.byref(st)), "maxent_fit")
    return theta[: (3 if nvdim == 1 else 10)], it.value, st.value


def maxwellian_grid(theta, sp, nvdim):
    """Ten-moment Maxwellian of Sec. 2.2 sampled at the velocity cell centres."""
    npts = sp.nv[0] if nvdim == 1 else sp.nv[0] * sp.nv[1] * sp.nv[2]
    out = np.zeros(npts)
    th = np.zeros(10)
    th[: len(theta)] = theta
    lib().or_maxwellian_grid(_d(th), ctypes.byref(sp), nvdim, _d(out))
    return out


def moment_fit(f, grid, sp, fluid, tol=1e-12, max_iter=20):
    """Moment fitting of Algorithm 1 (in place on f and fluid). Returns the
    stats (Newton iterations, fallbacks, clipped cells)."""
    stats = (ctypes.c_long * 3)(0, 0, 0)
    _check(lib().or_moment_fit(_d(f), ctypes.byref(grid), ctypes.byref(sp), _d(fluid), tol, max_iter,
                               ctypes.cast(stats, _lp)), "moment_fit")
    return tuple(stats)


def fluid_step(U, grid, sp, Q0, Qh, Q1, EB, dt):
    """One SSP-RK3 step of the ten-moment equations of Sec. 2.1 with CWENO
    fluxes and the third moment from f (in place on U)."""
    args = [np.ascontiguousarray(a, dtype=np.float64) for a in (Q0, Qh, Q1, EB)]
    _check(lib().or_fluid_step(_d(U), ctypes.byref(grid), ctypes.byref(sp), *[_d(a) for a in args], dt),
           "fluid_step")


CHI = 2.0 * math.sqrt(2.0 / math.pi)  # Sec. 2.3, after Hammett and Perkins


def closure_chi_k0(q, m, n0=1.0):
    """chi / k_s0 of the gradient closure (Sec. 2.3): k_s0 = 1/d_s with the
    inertial length d_s = sqrt(m_s / (mu0 n0 q_s^2)) at the reference
    density n0 of the normalisation (mu0 = 1)."""
    return CHI * math.sqrt(m / (n0 * q * q))


def fluid_step_closure(U, grid, sp, EB, dt, chi_k0):
    """One SSP-RK3 step of the stand-alone ten-moment fluid with the gradient
    heat-flux closure of Sec. 2.3 (in place on U; 2D3V)."""
    EB = np.ascontiguousarray(EB, dtype=np.float64)
    _check(lib().or_fluid_step_closure(_d(U), ctypes.byref(grid), ctypes.byref(sp), _d(EB), dt, chi_k0),
           "fluid_step_closure")


def fluid_rhs_closure(U, grid, sp, EB, chi_k0):
    """The semi-discrete right-hand side L(U) of the closure model."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    EB = np.ascontiguousarray(EB, dtype=np.float64)
    out = np.zeros_like(U)
    _check(lib().or_fluid_rhs_closure(_d(U), ctypes.byref(grid), ctypes.byref(sp), _d(EB), chi_k0, _d(out)),
           "fluid_rhs_closure")
    return out


def maxwellian_e3(u):
    """Third moment int v v v f of the closure model for one state
    (n, nu_a, E2_ab) (order xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(10)
    lib().or_maxwellian_e3(_d(u), _d(out))
    return out


def maxwell(yee, grid, J, h, c):
    """One FDTD leapfrog step of length h (Sec. 2.1; in place)."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    _check(lib().or_maxwell(_d(yee), ctypes.byref(grid), _d(J), h, c), "maxwell")


def fields_to_centres(yee, grid):
    EB = np.zeros((grid.nx * grid.ny, 6))
    lib().or_fields_to_centres(_d(yee), ctypes.byref(grid), _d(EB))
    return EB


def poisson_1d(rho, dx):
    """Periodic 1D Poisson solve dE/dx = rho (Sec. 3.1), E at cell centres."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    E = np.zeros_like(rho)
    lib().or_poisson_1d(_d(rho), rho.size, dx, _d(E))
    return E
