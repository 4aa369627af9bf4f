"""Host logic of bench.py's multi-GPU path (replicas: one independent run
per rank, the slowest rank's time, whole-job throughput; the reference arm
runs on rank 0 only), exercised with world_size-2 gloo process groups on the
CPU; and the arithmetic of the fit's ALU roofline from device counters."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.slowest(1.0 + 0.5 * rank, dist, "cpu")
    rate = bench.job_rate(1000, 4, world, t)
    out.put((rank, t, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_and_job_rate_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 1.5                      # the slower replica's time on every rank
        assert rate == 1000 * 4 * 2 / 1.5    # units of both replicas over that time


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest(2.5) == 2.5
    assert bench.job_rate(10, 3, 1, 2.0) == 15.0


def test_reference_arm_runs_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


@pytest.mark.slow
def test_reference_arm_prints_one_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


@pytest.mark.slow
def test_all_cores_oracle_figure():
    """The all-cores oracle figure: one spawned process per host core, each
    timing the same bounded sample; the aggregate counts every process's
    cells over the slowest process's time."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.cpu_all_cores("harris_512x256_v16", sample=(8, 4))
    assert r["kind"] == "oracle" and r["cores"] == (os.cpu_count() or 1) and r["value"] > 0
    assert "8x4" in r["sample"]


def test_newton_roofline_arithmetic():
    """The fit's ALU roofline from device counters (host arithmetic only):
    the method's work is 10 operations per velocity cell and moment
    evaluation and 25 more per Jacobian, over the phase time, against the
    measured FMA rate; the issued count weights the edge-start and the
    centre-out pass by the wide kernel's share of the fits; the DRAM
    traffic scales with the cells of one launch."""
    import bench
    from paper_2109_06743_gb300 import workloads as W
    cfg = W.named("harris_512x256_v16")
    n3 = 16 ** 3
    alu = {"fp32_tops": 40.0, "fp64_tops": 0.625}
    launches, fit_ms = 20, 200.0
    stats = [0] * 13
    stats[4], stats[5] = 2_000_000, 1_000_000  # moment and Jacobian evaluations
    r = bench.newton_roofline(cfg, stats, fit_ms, launches, alu)
    method = (10 * 2_000_000 + 25 * 1_000_000) * n3
    assert r["method_ops_per_launch"] == pytest.approx(method / launches)
    assert r["achieved"] == pytest.approx(method / 0.2 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 40.0) and r["method_frac"] == r["frac"]
    edge = (bench.ISSUED_OPS_MOMENT_EDGE * 2_000_000 + bench.ISSUED_OPS_GRAM_DF * 1_000_000) * n3
    assert r["issued_ops_per_launch"] == pytest.approx(edge / launches)
    assert r["issued_alu_ops_per_launch"] == pytest.approx(bench.ISSUED_ALU_OPS_MOMENT_EDGE * 2_000_000 * n3 / launches)
    assert r["traffic"] == pytest.approx(bench.NEWTON_DRAM_BYTES_PER_CELL[(False, 16)] * cfg.ncell)
    # every fit in the wide kernel: the centre-out count, no ALU-ordered sums
    stats[9] = 2 * cfg.ncell * launches
    w = bench.newton_roofline(cfg, stats, fit_ms, launches, alu)
    centre = (bench.ISSUED_OPS_MOMENT_CENTRE * 2_000_000 + bench.ISSUED_OPS_GRAM_DF * 1_000_000) * n3
    assert w["issued_ops_per_launch"] == pytest.approx(centre / launches)
    assert w["issued_alu_ops_per_launch"] == 0
    # the FP64 kernel's counters
    stats64 = [0] * 13
    stats64[10], stats64[11] = 2_000_000, 1_000_000
    f = bench.newton_roofline(cfg, stats64, fit_ms, launches, alu, fp64=True)
    assert f["peak"] == 0.625 and f["issued_ops_per_launch"] == pytest.approx((5 * 2_000_000 + 2 * 1_000_000) * n3 / launches)
