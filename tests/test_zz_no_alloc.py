"""mts_solve_static, the solve for callers that cannot allocate device memory when they
solve: it keeps its working state in the library's fixed device scratch instead of a
caller tape. Checked through the C ABI against mts_solve (+ mts_backward for dloss/dC) on
the same inputs, on two calls in a row, and for its size limit. Collected last on purpose
(file name) so that a stop-at-first-failure run has run every other test before it."""
import numpy as np
import pytest
import torch

from paper_2503_18479_gb300 import build_lib
from paper_2503_18479_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12  # same kernels and inputs as mts_solve: agreement to rounding


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _reference(sim, C, nv):
    """The existing entry points: mts_solve with a caller tape, then mts_backward."""
    ev = sim.make_eval(C, True)
    tape = sim.alloc_tape(C.shape[0])
    I = torch.empty((C.shape[0], sim.sumFN), dtype=torch.complex128, device="cuda")
    loss = torch.empty((C.shape[0], sim.n_struct), dtype=torch.float64, device="cuda")
    nv.mts_solve(sim.pb, sim.prec, sim.basis, ev, I, loss, tape)
    g = torch.empty((C.shape[0], sim.n_ports), dtype=torch.float64, device="cuda")
    ones = torch.ones((C.shape[0], sim.n_struct), dtype=torch.float64, device="cuda")
    nv.mts_backward(sim.pb, sim.prec, sim.basis, ev, tape, None, ones, g)
    return I, loss, g


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_static_solve_matches_mts_solve_twice(prec):
    assert torch.cuda.is_available()
    build_lib.build()
    from paper_2503_18479_gb300 import native as nv
    from paper_2503_18479_gb300.simulator import Simulator
    wl = W.array_8x8(seed=4, n_cfg=300, grid=16, planes=(0.02,))
    sim = Simulator(wl, prec)
    rng = np.random.Generator(np.random.PCG64(9))
    for call in range(2):
        C = torch.from_numpy(rng.uniform(20e-12, 200e-12, (300, 64))).cuda()
        I0, l0, g0 = _reference(sim, C, nv)
        ev = sim.make_eval(C, True)
        I1 = torch.empty_like(I0)
        l1 = torch.empty_like(l0)
        g1 = torch.empty_like(g0)
        nv.mts_solve_static(sim.pb, sim.prec, sim.basis, ev, I1, l1, g1)
        torch.cuda.synchronize()
        assert _rel(I1, I0) <= TOL, (call, _rel(I1, I0))
        assert _rel(l1, l0) <= TOL, (call, _rel(l1, l0))
        assert _rel(g1, g0) <= TOL, (call, _rel(g1, g0))


def test_static_solve_rejects_work_beyond_the_scratch():
    assert torch.cuda.is_available()
    build_lib.build()
    from paper_2503_18479_gb300 import native as nv
    from paper_2503_18479_gb300.simulator import Simulator
    wl = W.array_8x8(seed=1, n_cfg=2, grid=8, planes=(0.02,))
    sim = Simulator(wl, "mixed")
    limit = 32 << 20
    n_big = 1
    while nv.mts_tape_bytes(sim.pb, n_big, "mixed") <= limit:
        n_big *= 2
    C = torch.full((n_big, 64), 50e-12, dtype=torch.float64, device="cuda")
    with pytest.raises(nv.MtsError) as e:
        nv.mts_solve_static(sim.pb, sim.prec, sim.basis, sim.make_eval(C, True))
    assert e.value.code == nv.MTS_EWORKSPACE
