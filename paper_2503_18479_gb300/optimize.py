"""Gradient-descent fit of the capacitances (paper Sec. III-C: Adam, at most 2000 epochs,
learning rate 1e-13; Sec. V-B: clipping or tanh projection to a tuning range), run entirely
on the GPU: one epoch is mts_solve (currents, objective, adjoint dloss/dC at the loss
points) -> mts_backward (dloss/dC per configuration) -> mts_adam_step, captured once in a
CUDA graph and replayed. Every configuration of the batch is an independent fit (a batch of
initial values and/or targets, e.g. an initialisation sweep)."""
from __future__ import annotations

from typing import Optional

import torch

from . import native as nv
from .simulator import Simulator


class AdamFit:
    def __init__(self, sim: Simulator, C0: torch.Tensor, lr: float = 1e-13, betas=(0.9, 0.999),
                 eps: float = 1e-8, projection: Optional[str] = None, bounds=(0.0, 0.0),
                 max_epochs: int = 2000, use_graph: bool = True):
        if sim.target is None:
            raise ValueError("AdamFit needs a target (the objective's loss points)")
        dev = sim.device
        self.sim = sim
        self.n_cfg = C0.shape[0]
        self.C = C0.to(dev, torch.float64).contiguous().clone()
        self.opt = nv.MtsAdam(lr, betas[0], betas[1], eps, nv.PROJECTIONS[projection],
                              float(bounds[0]), float(bounds[1]))
        n = self.C.numel()
        self.u = None
        if projection == "tanh":
            mid, half = 0.5 * (bounds[1] + bounds[0]), 0.5 * (bounds[1] - bounds[0])
            z = ((self.C - mid) / half).clamp(-1 + 1e-12, 1 - 1e-12)
            self.u = torch.atanh(z).contiguous()
            self.C = (mid + half * torch.tanh(self.u)).contiguous()
        self.m = torch.zeros(n, dtype=torch.float64, device=dev)
        self.v = torch.zeros(n, dtype=torch.float64, device=dev)
        self.step = torch.zeros(1, dtype=torch.int64, device=dev)
        self.ev = sim.make_eval(self.C, True)
        self.tape = sim.alloc_tape(self.n_cfg)
        self.loss = torch.empty((self.n_cfg, sim.n_struct), dtype=torch.float64, device=dev)
        self.grad = torch.empty((self.n_cfg, sim.n_ports), dtype=torch.float64, device=dev)
        self.ones = torch.ones((self.n_cfg, sim.n_struct), dtype=torch.float64, device=dev)
        self.history = torch.full((max_epochs, self.n_cfg, sim.n_struct), float("nan"),
                                  dtype=torch.float64, device=dev)
        self.max_epochs = max_epochs
        self.use_graph = use_graph
        self.graph = None

    def _epoch(self, stream=None):
        s = self.sim
        nv.mts_solve(s.pb, s.prec, s.basis, self.ev, None, self.loss, self.tape, stream)
        nv.mts_backward(s.pb, s.prec, s.basis, self.ev, self.tape, None, self.ones, self.grad, stream)
        nv.mts_adam_step(self.C.numel(), self.opt, self.C, self.u, self.grad, self.m, self.v,
                         self.step, self.loss, self.history, stream)

    def _capture(self):
        side = torch.cuda.Stream(device=self.sim.device)
        side.wait_stream(torch.cuda.current_stream(self.sim.device))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            self._epoch()
        torch.cuda.current_stream(self.sim.device).wait_stream(side)
        return g

    def run(self, epochs: int):
        """Run `epochs` Adam epochs (at most max_epochs in all); returns (C, history) where
        history[e] is the objective at the start of epoch e (NaN beyond the epochs run)."""
        done = int(self.step.item())
        epochs = min(epochs, self.max_epochs - done)
        if self.use_graph and epochs > 1:
            if self.graph is None:
                self._epoch()  # one eager epoch first (kernel attributes, lazy loads)
                epochs -= 1
                self.graph = self._capture()
            for _ in range(epochs):
                self.graph.replay()
        else:
            for _ in range(epochs):
                self._epoch()
        torch.cuda.synchronize(self.sim.device)
        return self.C, self.history
