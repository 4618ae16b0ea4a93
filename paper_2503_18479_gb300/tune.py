"""Autotuner of the launch schedule: times the forward step (mts_solve + mts_superpose) of a
Simulator on a given batch for each candidate schedule and keeps the fastest in
`sim.tuning` (passed to every later call through mts_eval). The candidates choose, per
structure, the tensor-core or the SIMT superposition (the threshold on configurations x
frequencies), the CTA size of the blocked solve for N > 64 (128, 256 or 512 threads per
system; with MTS_MIXED / MTS_BF16 and at most 128 ports, 256 and 512 also keep the matrix in
shared memory, one system per SM), and whether the register classes of up to 32 ports run one mapping wider (a half
warp, a warp or a two-warp CTA per system instead of the class's own). Every schedule
computes the same result to rounding; only time differs."""
from __future__ import annotations

import itertools

import torch

from . import native as nv
from .simulator import Simulator

SIMT_CHOICES = (-1, 4, 16, 64, 1 << 30)  # -1: every structure on the tensor cores
LARGE_CHOICES = (128, 256, 512)
WIDEN_CHOICES = (1, 2, 4, 7)  # register classes run one mapping wider (bit c: class c)


def _time_step(sim: Simulator, C: torch.Tensor, tuning: dict, reps: int, flush: torch.Tensor):
    saved = sim.tuning
    sim.tuning = tuning
    try:
        ev = sim.make_eval(C, sim.target is not None)
        n = C.shape[0]
        tape = sim.alloc_tape(n)
        B = torch.empty((n, sim.sumFP), dtype=sim.b_dtype, device=sim.device)
        loss = None if sim.target is None else torch.empty((n, sim.n_struct), dtype=torch.float64,
                                                           device=sim.device)
        st = torch.cuda.current_stream(sim.device)

        def step():
            nv.mts_solve(sim.pb, sim.prec, sim.basis, ev, None, loss, tape)
            nv.mts_superpose(sim.pb, sim.prec, sim.basis, ev, tape, B)

        step()
        torch.cuda.synchronize(sim.device)
        best = float("inf")
        for _ in range(reps):
            flush.fill_(1)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(st)
            step()
            a1.record(st)
            a1.synchronize()
            best = min(best, a0.elapsed_time(a1))
        return best
    finally:
        sim.tuning = saved


def autotune(sim: Simulator, C: torch.Tensor, reps: int = 3):
    """Time every candidate schedule on this batch; set and return the fastest
    (sim.tuning) together with all timings in ms."""
    C = C.to(sim.device, torch.float64).contiguous()
    has_large = any(st.n_ports > 64 for st in sim.wl.structures)
    simt = SIMT_CHOICES if sim.prec != nv.MTS_FP64 else (0,)
    large = LARGE_CHOICES if has_large else (0,)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=sim.device)
    times = {}
    for s_thr, l_thr in itertools.product(simt, large):
        tuning = {"simt_max_sys": s_thr, "large_threads": l_thr, "reg_widen": 0}
        times[(s_thr, l_thr, 0)] = _time_step(sim, C, tuning, reps, flush)
    best = min(times, key=times.get)
    # then, with that pair, the mapping of the register classes present (warp-per-system
    # against wider groups of threads per system)
    classes = {0 if n <= 8 else 1 if n <= 16 else 2 for n in (st.n_ports for st in sim.wl.structures)
               if n <= 32}
    for w in WIDEN_CHOICES:
        if any((w >> c) & 1 for c in classes):
            tuning = {"simt_max_sys": best[0], "large_threads": best[1], "reg_widen": w}
            times[(best[0], best[1], w)] = _time_step(sim, C, tuning, reps, flush)
    best = min(times, key=times.get)
    sim.tuning = {"simt_max_sys": best[0], "large_threads": best[1], "reg_widen": best[2]}
    return sim.tuning, times
