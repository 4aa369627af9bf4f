"""The production-run module on a small named workload: JSON lines with the
energy partition, drift, masses, reconnected flux and rate, step time and
Newton iterations; online retraining of the warm-start network runs and
leaves the fits converging (no fallbacks)."""
import json

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2109_06743_gb300 import build
    build.build()
    return torch


def test_run_module_lines_and_retraining(gpu, tmp_path):
    from paper_2109_06743_gb300 import run
    out = tmp_path / "run.jsonl"
    assert run.main(["--workload", "asym_256x128_v12", "--steps", "6", "--every", "3", "--retrain-every", "4",
                     "--out", str(out)]) == 0
    lines = [json.loads(x) for x in out.read_text().splitlines()]
    assert len(lines) == 3 and lines[0]["mlp"] and len(lines[0]["channels"]) == 4
    for ln in lines[1:]:
        assert abs(sum(ln["energy_fraction"]) - 1.0) < 1e-12
        assert abs(ln["energy_drift"]) < 1e-4
        assert max(abs(m) for m in ln["mass_rel_change"]) < 1e-5
        assert ln["ms_per_step"] > 0 and 1.0 <= ln["newton_iterations_per_fit"] < 4.0
        assert ln["slow_evaluations_per_fit"] == 0.0 and ln["newton_fallbacks"] == 0
    assert lines[1]["retrains"] == 0 and lines[2]["retrains"] == 1
    assert lines[2]["step"] == 6 and abs(lines[2]["t"] - 6 * lines[0]["dt"]) < 1e-15
