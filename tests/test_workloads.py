"""Pins of the synthetic input generators: the asymmetric sheet is in exact
pressure balance with the stated far fields, its magnetic field is
discretely divergence free, and the counter-hash noise is reproducible; the
configuration's JSON form (checkpoints) round-trips."""
import numpy as np
import pytest

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


def test_training_schedule_covers_every_step(monkeypatch):
    """warmstart._train splits the Adam steps into the segments of
    LR_SCHEDULE in order: the segments add up to the requested steps, each
    runs at lr times its factor with its own seed, and the losses of all
    steps come back in order (host logic; the training call is stubbed)."""
    import numpy as np
    from paper_2109_06743_gb300 import abi, warmstart
    calls = []

    def fake_train(ctx, buf, n, steps, batch=4096, lr=1e-3, seed=0, record_loss=False, stream=None):
        calls.append((steps, lr, seed))
        start = sum(c[0] for c in calls[:-1])
        return np.arange(start, start + steps, dtype=float)

    monkeypatch.setattr(abi, "mlp_train", fake_train)
    for total in (3000, 10000, 7, 1):
        calls.clear()
        losses = warmstart._train(None, None, 1, total, 4096, 2e-3, 100, None)
        assert sum(c[0] for c in calls) == total
        assert np.array_equal(losses, np.arange(total, dtype=float))
        factors = [f for _, f in warmstart.LR_SCHEDULE]
        assert all(c[0] > 0 for c in calls)
        used = [(s, lr) for s, lr, _ in calls]
        # the rates never rise and start at lr
        assert used[0][1] == 2e-3 and all(a[1] >= b[1] for a, b in zip(used, used[1:]))
        assert len({c[2] for c in calls}) == len(calls)
    calls.clear()
    warmstart._train(None, None, 1, 3000, 4096, 2e-3, 100, None)
    assert [c[0] for c in calls] == [1500, 1000, 500]
    assert np.allclose([c[1] for c in calls], [2e-3 * f for f in factors])
    assert W.TRAIN_STEPS.get("asym_256x128_v12") == 10000 and "harris_128x64_v16" not in W.TRAIN_STEPS


@pytest.mark.parametrize("make", [lambda: W.landau(), lambda: W.two_stream(precision=32),
                                  lambda: W.named("harris_128x64_v20", precision=64),
                                  lambda: W.named("harris_512x256_v16", sub=(64, 32)),
                                  lambda: W.named("asym_1024x512_v12")])
def test_config_json_round_trip(make):
    """checkpoints store the configuration as JSON: every field and every
    attribute the builders add comes back"""
    cfg = make()
    cfg.fit_tol = 3e-12
    back = W.config_from_json(W.config_to_json(cfg))
    assert back == cfg and vars(back) == vars(cfg)
    for a, b in zip(back.species, cfg.species):
        assert vars(a) == vars(b) and isinstance(a.nv, tuple) and a.dv == b.dv
    assert back.phase_cells() == cfg.phase_cells()
