"""Checkpoint and resume, and the per-step diagnostics log.

* A Simulation saved after some steps and resumed from the file continues
  bit for bit as the uninterrupted run: f, fluid state, Yee and cell-centred
  fields and the moments at t equal after the remaining steps. Cases: the
  FP32 Harris sheet with the network warm start (the network's parameters
  travel in the checkpoint), the Harris sheet with fitting off (standard
  PFC), and the 1D1V Landau run (Poisson field, Strang splitting).
* ``run(steps, log=...)`` writes one JSON line per logged step; the lines
  carry the step number, conserved masses and the same energy total as
  ``total_energy()``.
"""
import json

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


def _network(cfg, torch):
    """parameters of a network with a real input standardisation (samples
    harvested from two steps of the same sheet) and random weights"""
    from paper_2109_06743_gb300 import abi
    from paper_2109_06743_gb300.driver import Simulation
    sim = Simulation(cfg, W.harris_state(cfg, dtype=np.float32), None, W.harris_yee(cfg))
    cap = 40000
    buf = torch.zeros((cap, abi.MLP_SAMPLE), dtype=torch.float32, device="cuda")
    abi.mlp_set_harvest(sim.ctx, buf, cap, sim.stream)
    for _ in range(2):
        sim.step()
    n = abi.mlp_harvest_count(sim.ctx, sim.stream)
    abi.mlp_set_harvest(sim.ctx, None, 0, sim.stream)
    abi.mlp_init(sim.ctx, 5)
    abi.mlp_normalize(sim.ctx, buf, n, sim.stream)
    w = abi.mlp_get_weights(sim.ctx)
    sim.close()
    return w


def _same(a, b, torch):
    b.stream.synchronize()
    a.stream.synchronize()
    for x, y in zip(a.f, b.f):
        assert torch.equal(x, y)
    for x, y in zip(a.mom_t, b.mom_t):
        assert torch.equal(x, y)
    assert torch.equal(a.fluid, b.fluid) and torch.equal(a.eb, b.eb)
    if a.yee is not None:
        assert torch.equal(a.yee, b.yee)
    assert a.time == b.time and a.nstep == b.nstep


@pytest.mark.parametrize("case", ["harris_warm", "harris_standard_pfc", "landau"])
def test_resume_continues_bit_for_bit(gpu, tmp_path, case):
    from paper_2109_06743_gb300 import abi
    from paper_2109_06743_gb300.driver import Simulation
    torch = gpu
    if case == "landau":
        cfg = W.landau(nx=32, nv=32, precision=64)
        make = lambda: Simulation(cfg, W.landau_state(cfg))  # noqa: E731
        first, rest, use_mlp = 6, 6, False
    else:
        cfg = W.harris(nx=16, ny=8, nv=8, lx=3.2, ly=1.6, precision=32)
        fit = case == "harris_warm"
        make = lambda: Simulation(cfg, W.harris_state(cfg, dtype=np.float32), None, W.harris_yee(cfg), fit=fit)  # noqa: E731
        first, rest, use_mlp = 3, 3, fit
    w = _network(cfg, torch) if use_mlp else None
    a = make()
    b = make()
    for s in (a, b):
        if w is not None:
            abi.mlp_set_weights(s.ctx, w)
    for _ in range(first):
        a.step(use_mlp=use_mlp)
        b.step(use_mlp=use_mlp)
    path = str(tmp_path / "state.npz")
    b.save(path)
    b.close()
    c = Simulation.resume(path)
    assert c.cfg == cfg and vars(c.cfg) == vars(cfg)
    if w is not None:
        assert np.array_equal(abi.mlp_get_weights(c.ctx), w)
    for _ in range(rest):
        a.step(use_mlp=use_mlp)
        c.step(use_mlp=use_mlp)
    _same(a, c, torch)
    if use_mlp:
        assert abi.vl_read_stats(c.ctx)[12] > 0  # the resumed run used the network
    a.close()
    c.close()


def test_run_writes_one_json_line_per_logged_step(gpu, tmp_path):
    from paper_2109_06743_gb300.driver import Simulation
    cfg = W.harris(nx=16, ny=8, nv=12, lx=3.2, ly=1.6, precision=64)
    sim = Simulation(cfg, W.harris_state(cfg), None, W.harris_yee(cfg))
    path = tmp_path / "run.jsonl"
    sim.run(5, log=str(path), every=2)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert [d["step"] for d in lines] == [2, 4, 5]
    for d in lines:
        assert {"time", "mass", "kinetic_thermal", "electric", "magnetic", "total_energy", "reconnected_flux",
                "newton_iterations", "newton_fallbacks", "clipped_cells", "ms_per_step"} <= set(d)
        assert d["newton_iterations"] > 0 and d["ms_per_step"] > 0
        assert d["invalid_fits"] == 0
    m0 = np.array(lines[0]["mass"])
    for d in lines[1:]:
        np.testing.assert_allclose(d["mass"], m0, rtol=1e-12)
    assert lines[-1]["total_energy"] == pytest.approx(sim.total_energy(), rel=1e-15)
    assert lines[-1]["time"] == pytest.approx(5 * cfg.dt)
    sim.close()


def test_production_run_resumes_from_its_checkpoint(gpu, tmp_path):
    """run.py: four steps in one go and two steps, a checkpoint, and two more
    steps resumed from it end in the same checkpoint, array by array"""
    from paper_2109_06743_gb300 import run
    straight, split = str(tmp_path / "straight.npz"), str(tmp_path / "split.npz")
    log = tmp_path / "resumed.jsonl"
    common = ["--workload", "harris_128x64_v16", "--every", "2", "--no-mlp"]
    assert run.main(common + ["--steps", "4", "--save", straight]) == 0
    assert run.main(common + ["--steps", "2", "--save", split]) == 0
    assert run.main(["--resume", split, "--steps", "2", "--every", "2", "--no-mlp", "--save", split,
                     "--out", str(log)]) == 0
    za, zb = np.load(straight), np.load(split)
    assert sorted(za.files) == sorted(zb.files)
    for name in za.files:
        assert np.array_equal(za[name], zb[name]), name
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert lines[0]["step"] == 2 and lines[-1]["step"] == 4
