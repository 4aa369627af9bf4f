"""Training of the moment-fit warm-start network on the fits of a
cold-started run (the learned part of the moment fit: the network maps a
cell's target moments to a warm start of its Newton fit, Sec. 2.2 with
Algorithm 1's fit). The samples are harvested by the Newton kernel from its
converged fits; normalisation, training (BF16 tensor-core GEMMs, FP32
accumulation, Adam) and inference run in the library's kernels."""
import math
import time

import numpy as np
import torch

from . import abi
from . import workloads as W
from .driver import Simulation


# learning-rate schedule of the training: (share of the Adam steps, factor
# of the learning rate), in order. A stepped decay over the last half
# (measured on the asymmetric sheet, three seeds each: fit time 3.44-3.49 ms
# per step at 256 x 128 against 3.44-3.71 ms with a constant rate)
LR_SCHEDULE = ((0.5, 1.0), (1.0 / 3.0, 0.3), (1.0 / 6.0, 0.1))


def _train(ctx, buf, n, train_steps, batch, lr, seed, stream):
    """Adam steps in the segments of LR_SCHEDULE (segment ends at the
    cumulative shares, rounded up, so that a short run starts at the full
    rate); the losses of every step."""
    losses = []
    done, cum = 0, 0.0
    for k, (share, factor) in enumerate(LR_SCHEDULE):
        cum += share
        end = train_steps if k == len(LR_SCHEDULE) - 1 else min(train_steps, math.ceil(cum * train_steps - 1e-9))
        steps = end - done
        if steps > 0:
            losses += list(abi.mlp_train(ctx, buf, n, steps, batch=batch, lr=lr * factor, seed=seed + k,
                                         record_loss=True, stream=stream))
        done = max(done, end)
    return np.asarray(losses)


def train_warm_start(name, device, harvest_steps=24, train_steps=None, batch=4096, lr=2e-3):
    """Harvest (inputs, eta* - eta_0) samples from the converged fits of
    harvest_steps cold-started steps of the named workload, train the
    warm-start network on the GPU with the project's own kernels (Adam,
    train_steps steps, by default workloads.TRAIN_STEPS of the run or 3000;
    learning rate lr stepped down by LR_SCHEDULE), and return its weights
    and a summary (sample count, first and last losses, seconds)."""
    t0 = time.perf_counter()
    if train_steps is None:
        train_steps = W.TRAIN_STEPS.get(name, 3000)
    cfg = W.named(name, precision=32)
    sim = Simulation(cfg, W.initial_state(cfg, np.float32), None, W.initial_yee(cfg), device=device)
    cap = harvest_steps * 4 * cfg.ncell
    buf = torch.zeros((cap, abi.MLP_SAMPLE), dtype=torch.float32, device=device)
    abi.mlp_set_harvest(sim.ctx, buf, cap, sim.stream)
    for _ in range(harvest_steps):
        sim.step()
    n = abi.mlp_harvest_count(sim.ctx, sim.stream)
    abi.mlp_set_harvest(sim.ctx, None, 0, sim.stream)
    abi.mlp_init(sim.ctx, 2109)
    abi.mlp_normalize(sim.ctx, buf, n, sim.stream)
    t1 = time.perf_counter()
    losses = _train(sim.ctx, buf, n, train_steps, batch, lr, 6743, sim.stream)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    w = abi.mlp_get_weights(sim.ctx)
    sim.close()
    del buf
    info = {"trained_on": "%s, %d cold-started steps" % (name, harvest_steps), "samples": int(n),
            "train_steps": train_steps, "batch": batch, "lr": lr, "lr_schedule": [list(x) for x in LR_SCHEDULE],
            "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-20:])),
            "harvest_seconds": t1 - t0, "train_seconds": t2 - t1}
    return w, info


def retrain(sim, train_steps=1500, batch=4096, lr=2e-3, seed=2109, use_mlp=True):
    """Retrain the warm-start network of a running simulation on the fits of
    its next step (one step is run with the harvest on): the network is
    re-initialised, standardised on the new samples and trained, so that
    it follows the cells' moments as the run leaves the states it was
    trained on. Returns a summary (sample count, last loss, seconds)."""
    cfg = sim.cfg
    t0 = time.perf_counter()
    cap = 4 * cfg.ncell
    buf = torch.zeros((cap, abi.MLP_SAMPLE), dtype=torch.float32, device=sim.dev)
    abi.mlp_set_harvest(sim.ctx, buf, cap, sim.stream)
    sim.step(use_mlp=use_mlp)
    n = abi.mlp_harvest_count(sim.ctx, sim.stream)
    abi.mlp_set_harvest(sim.ctx, None, 0, sim.stream)
    abi.mlp_init(sim.ctx, seed)
    abi.mlp_normalize(sim.ctx, buf, n, sim.stream)
    losses = _train(sim.ctx, buf, n, train_steps, batch, lr, seed + 1, sim.stream)
    torch.cuda.synchronize()
    del buf
    return {"samples": int(n), "loss_last": float(np.mean(losses[-20:])), "seconds": time.perf_counter() - t0}
