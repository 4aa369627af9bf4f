"""Helpers for the GPU parity tests: run single C-ABI calls of libvlasov on
numpy inputs and read the results back. Inputs come from
paper_2109_06743_gb300.workloads (seeded); expected values come from the
oracle only."""
from __future__ import annotations

import numpy as np

from paper_2109_06743_gb300 import abi


class AbiRunner:
    """A context over explicit numpy state: f per species, fluid, Yee, eb."""

    def __init__(self, cfg, f_list, fluid=None, yee=None, eb=None):
        import torch
        self.torch = torch
        self.cfg = cfg
        dev = torch.device("cuda:0")
        self.dev = dev
        dt = torch.float32 if cfg.precision == 32 else torch.float64
        nc = cfg.ncell
        self.ncomp = 3 if cfg.nvdim == 1 else 10
        self.nmom = 4 if cfg.nvdim == 1 else 20
        self.f = [torch.as_tensor(np.ascontiguousarray(f).reshape(nc, -1)).to(dev, dt).contiguous() for f in f_list]
        ns = len(cfg.species)
        fl = np.zeros((ns, nc, self.ncomp)) if fluid is None else np.asarray(fluid, dtype=np.float64)
        self.fluid = torch.as_tensor(np.ascontiguousarray(fl.reshape(ns, nc, self.ncomp))).to(dev).contiguous()
        e = np.zeros((nc, 6)) if eb is None else np.asarray(eb, dtype=np.float64)
        self.eb = torch.as_tensor(np.ascontiguousarray(e.reshape(nc, 6))).to(dev).contiguous()
        if cfg.nvdim == 3:
            y = np.zeros((6, cfg.ny + 1, cfg.nx)) if yee is None else np.asarray(yee, dtype=np.float64)
            self.yee = torch.as_tensor(np.ascontiguousarray(y.reshape(-1))).to(dev).contiguous()
        else:
            self.yee = None
        self.desc = abi.make_desc(cfg)
        nb = abi.vlasov_work_bytes(self.desc)
        assert nb > 0, abi.lib().vl_last_error(None)
        self.work = torch.zeros(nb + 256, dtype=torch.uint8, device=dev)
        off = (-self.work.data_ptr()) % 256
        self.ctx = abi.vlasov_init(self.desc, self.f, self.fluid, self.yee, self.eb, self.work.data_ptr() + off, nb)
        self.stream = torch.cuda.current_stream(dev)

    def mom(self):
        return self.torch.zeros((self.cfg.ncell, self.nmom), dtype=self.torch.float64, device=self.dev)

    def sync(self):
        self.torch.cuda.synchronize()

    def f_np(self, k):
        self.sync()
        return self.f[k].double().cpu().numpy()

    def close(self):
        abi.vlasov_free(self.ctx)
