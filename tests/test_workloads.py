"""Pins of the synthetic input generators: the asymmetric sheet is in exact
pressure balance with the stated far fields, its magnetic field is
discretely divergence free, and the counter-hash noise is reproducible."""
import numpy as np

from paper_2109_06743_gb300 import workloads as W


def test_asymmetric_sheet_pressure_balance_and_far_fields():
    cfg = W.asym_sheet(nx=8, ny=8, nv=8, lx=3.2, ly=6.4)
    y = np.linspace(-20, 20, 401)
    n, tt, bx = W.asym_profiles(cfg, y)
    p = n * tt + 0.5 * bx * bx
    assert np.allclose(p, p[0], rtol=0, atol=1e-13)
    assert abs(n[0] / n[-1] - 10.0) < 1e-9 and abs(tt[-1] / tt[0] - 3.0) < 1e-9
    assert abs(bx[-1] - 1.0) < 1e-9 and bx[0] < 0 and np.all(n > 0)


def test_asymmetric_yee_divergence_free_and_reproducible():
    cfg = W.asym_sheet(nx=12, ny=10, nv=8, lx=3.2, ly=6.4)
    y1, y2 = W.asym_yee(cfg), W.asym_yee(cfg)
    assert np.array_equal(y1, y2)
    bx, by = y1[3], y1[4]
    # div B at cell centres of the corner grid: dBx/dx + dBy/dy = 0 (periodic x)
    div = (np.roll(bx[:cfg.ny], -1, axis=1) - bx[:cfg.ny]) / cfg.dx + (by[1:] - by[:-1]) / cfg.dy
    assert np.abs(div).max() < 1e-10 * np.abs(bx).max() / cfg.dx
    assert np.all(y1[5][:cfg.ny] == cfg.bguide)
