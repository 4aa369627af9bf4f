"""GPU parity and usefulness of the moment-fit warm-start network.

* forward: the tensor-core BF16 network against the FP64 oracle network on
  the same (FP32) parameters and inputs. BF16 keeps 8 significant bits
  (unit roundoff 2^-9 ~ 2e-3) on the standardised inputs, the weights and the
  hidden activations; summed over 128 terms with random signs the outputs
  carry ~1e-2 of their spread: bound 3e-2 of the output spread (RMS) and
  1e-1 elementwise.
* gradients: same arithmetic plus the BF16 backward operands: each parameter
  block within 5e-2 (relative norm) of the oracle's chain-rule gradient, the
  loss within 1e-2.
* training decreases the loss, and a network trained on samples harvested
  from Harris-sheet fits lowers the mean Newton iteration count of held-out
  fits while the fitted Maxwellians stay those of the cold start (Newton
  runs to the same tolerance).
"""
import numpy as np
import pytest

from paper_2109_06743_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2109_06743_gb300 import build
    build.build()
    return torch


def _runner(nv=8):
    from gpu_util import AbiRunner
    cfg = W.harris(nx=4, ny=4, nv=nv, lx=0.8, ly=0.8, precision=32)
    f0 = [W.random_blocks((cfg.ncell, nv ** 3), 40 + k) for k in range(2)]
    return AbiRunner(cfg, f0)


def _random_blob(rng):
    from oracle import mlp as M
    p = {"xm": rng.normal(size=12) * 0.2, "xs": 0.5 + rng.uniform(size=12),
         "ym": rng.normal(size=10) * 0.1, "ys": 0.2 + rng.uniform(size=10), "ysc": 10.0 ** rng.uniform(-5, -2, size=10),
         "W1": rng.normal(size=(128, 12)) * 0.4, "b1": rng.normal(size=128) * 0.1,
         "W2": rng.normal(size=(128, 128)) * 0.12, "b2": rng.normal(size=128) * 0.1,
         "W3": rng.normal(size=(10, 128)) * 0.12, "b3": rng.normal(size=10) * 0.1}
    return M.pack(p).astype(np.float32)


def test_forward_matches_oracle(gpu):
    from oracle import mlp as M
    from paper_2109_06743_gb300 import abi
    torch = gpu
    r = _runner()
    rng = np.random.default_rng(11)
    w = _random_blob(rng)
    abi.mlp_set_weights(r.ctx, w)
    n = 1000  # not a multiple of the 128-sample tile
    x = (rng.normal(size=(n, 12)) * 1.5).astype(np.float32)
    xd = torch.as_tensor(x, device="cuda")
    yd = torch.zeros((n, 10), dtype=torch.float32, device="cuda")
    abi.mlp_forward(r.ctx, xd, n, yd)
    t = yd.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(t))
    # compare in the network's own output space, y = (asinh(t / ysc) - ym) / ys
    p = M.unpack(w.astype(np.float64))
    y = (np.arcsinh(t / p["ysc"]) - p["ym"]) / p["ys"]
    ref = M._layers(p, x.astype(np.float64))[-1]
    spread = np.sqrt(np.mean((ref - ref.mean(axis=0)) ** 2, axis=0))
    rms = np.sqrt(np.mean((y - ref) ** 2, axis=0)) / spread
    assert np.all(rms <= 3e-2), rms
    assert np.all(np.abs(y - ref) <= 1e-1 * spread), float(np.max(np.abs(y - ref) / spread))
    # and t itself where the transform is nearly linear
    small = np.abs(ref * p["ys"] + p["ym"]) < 0.5
    tref = M.forward(w.astype(np.float64), x.astype(np.float64))
    assert np.all(np.abs(t - tref)[small] <= 0.1 * (p["ysc"] * p["ys"] * spread)[np.newaxis, :].repeat(len(t), 0)[small])
    # NaN inputs give NaN outputs (never a usable prediction)
    abi.mlp_forward(r.ctx, torch.full((3, 12), float("nan"), device="cuda"), 3, yd)
    assert torch.isnan(yd[:3]).all()
    r.close()


def test_gradient_matches_oracle(gpu):
    from oracle import mlp as M
    from paper_2109_06743_gb300 import abi
    torch = gpu
    r = _runner()
    rng = np.random.default_rng(12)
    w = _random_blob(rng)
    abi.mlp_set_weights(r.ctx, w)
    n = 300
    s = np.zeros((n, abi.MLP_SAMPLE), dtype=np.float32)
    s[:, :12] = rng.normal(size=(n, 12)) * 1.5
    s[:, 12:22] = rng.normal(size=(n, 10)) * 10.0 ** rng.uniform(-5, -2, size=(n, 10))
    s[:, 22] = 1.0
    sd = torch.as_tensor(s, device="cuda")
    gd = torch.zeros(abi.MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = abi.mlp_grad(r.ctx, sd, n, gd)
    g = gd.cpu().numpy().astype(np.float64)
    lref, gref = M.loss_and_grad(w.astype(np.float64), s.astype(np.float64))
    assert abs(loss - lref) <= 1e-2 * lref, (loss, lref)
    P, R = M.unpack(g), M.unpack(gref)
    for name in M.TRAINED:
        err = np.linalg.norm(P[name] - R[name]) / np.linalg.norm(R[name])
        assert err <= 5e-2, (name, err)
    for name in ("xm", "xs", "ym", "ys", "ysc"):
        assert np.all(P[name] == 0)
    r.close()


def test_training_reduces_loss(gpu):
    from paper_2109_06743_gb300 import abi
    torch = gpu
    r = _runner()
    rng = np.random.default_rng(13)
    n = 20000
    x = rng.normal(size=(n, 12))
    A = rng.normal(size=(12, 10)) / np.sqrt(12)
    s = np.zeros((n, abi.MLP_SAMPLE), dtype=np.float32)
    s[:, :12] = x
    s[:, 12:22] = np.tanh(x @ A) + 0.3 * np.sin(x[:, :10])
    s[:, 22] = 1.0
    sd = torch.as_tensor(s, device="cuda")
    abi.mlp_init(r.ctx, 5)
    abi.mlp_normalize(r.ctx, sd, n)
    losses = abi.mlp_train(r.ctx, sd, n, steps=300, batch=1024, lr=2e-3, seed=9, record_loss=True)
    first, last = np.mean(losses[:10]), np.mean(losses[-10:])
    assert np.all(np.isfinite(losses))
    assert last < 0.1 * first, (first, last)
    r.close()


def _fit_part_of_step(sim, dt):
    """Algorithm 1 up to (not including) the moment fit, as driver.step does."""
    from paper_2109_06743_gb300 import abi
    ctx, s = sim.ctx, sim.stream
    abi.maxwell_step(ctx, 0.5 * dt, None, s)
    for k in range(len(sim.cfg.species)):
        abi.pfc_advect_x(ctx, k, 0, dt, s)
        abi.pfc_advect_x(ctx, k, 1, dt, s)
        abi.pfc_advect_v(ctx, k, dt, sim.mom_t1[k], s)
    abi.fluid_step(ctx, dt, sim.mom_t, sim.mom_t1, s)


def test_warm_start_lowers_newton_iterations(gpu):
    from paper_2109_06743_gb300 import abi
    from paper_2109_06743_gb300.driver import Simulation
    torch = gpu
    cfg = W.harris(nx=32, ny=16, nv=12, lx=6.4, ly=3.2, precision=32)
    sim = Simulation(cfg, W.harris_state(cfg, dtype=np.float32), None, W.harris_yee(cfg))
    cap = 200000
    buf = torch.zeros((cap, abi.MLP_SAMPLE), dtype=torch.float32, device="cuda")
    abi.mlp_set_harvest(sim.ctx, buf, cap, sim.stream)
    for _ in range(20):
        sim.step()
    n = abi.mlp_harvest_count(sim.ctx, sim.stream)
    abi.mlp_set_harvest(sim.ctx, None, 0, sim.stream)
    assert n > 20000
    abi.mlp_init(sim.ctx, 21)
    abi.mlp_normalize(sim.ctx, buf, n, sim.stream)
    losses = abi.mlp_train(sim.ctx, buf, n, steps=1500, batch=2048, lr=2e-3, seed=3, record_loss=True,
                           stream=sim.stream)
    assert np.mean(losses[-20:]) < 0.2 * np.mean(losses[:20]), (np.mean(losses[:20]), np.mean(losses[-20:]))
    for _ in range(3):
        sim.step()  # held-out states
    _fit_part_of_step(sim, cfg.dt)
    nc = cfg.ncell
    iters = {}
    for k in range(len(cfg.species)):
        fluid0 = sim.fluid[k].clone()
        th = {}
        for warm in (0, 1):
            sim.fluid[k].copy_(fluid0)
            tv = torch.zeros((nc, 10), dtype=torch.float64, device="cuda")
            tf = torch.zeros((nc, 10), dtype=torch.float64, device="cuda")
            abi.vl_reset_stats(sim.ctx, sim.stream)
            abi.moment_fit_solve(sim.ctx, k, sim.mom_t1[k], warm, tv, tf, sim.stream)
            st = abi.vl_read_stats(sim.ctx, sim.stream)
            iters[(k, warm)] = st[0] / (2.0 * nc)
            assert st[3] == 0
            th[warm] = (tv.cpu().numpy(), tf.cpu().numpy())
        for a, b in zip(th[0], th[1]):
            scale = np.abs(a).max(axis=0, keepdims=True) + 1e-300
            assert np.all(np.abs(a - b) <= 1e-8 * scale), float(np.max(np.abs(a - b) / scale))
    cold = np.mean([iters[(k, 0)] for k in range(2)])
    warm = np.mean([iters[(k, 1)] for k in range(2)])
    print("Newton iterations per fit: cold %.3f, warm %.3f" % (cold, warm))
    assert warm < 0.85 * cold, (cold, warm)
    sim.close()
