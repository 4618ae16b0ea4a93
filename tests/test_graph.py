"""The whole step (solve + objective + adjoint, superposition, gradient combine) captured in
one CUDA graph and replayed on new capacitances: the ABI allocates nothing and never
synchronises, so a replay must give exactly the eager results."""
import numpy as np
import pytest
import torch

from helpers import small_8x8, small_ragged
from paper_2503_18479_gb300 import build_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    build_lib.build()


def _buffers(sim, n):
    return dict(tape=sim.alloc_tape(n),
                B=torch.empty((n, sim.sumFP), dtype=sim.b_dtype, device="cuda"),
                loss=torch.empty((n, sim.n_struct), dtype=torch.float64, device="cuda"),
                g=torch.empty((n, sim.n_ports), dtype=torch.float64, device="cuda"),
                gl=torch.ones((n, sim.n_struct), dtype=torch.float64, device="cuda"))


def _step(nv, sim, ev, b):
    nv.mts_solve(sim.pb, sim.prec, sim.basis, ev, None, b["loss"], b["tape"])
    nv.mts_superpose(sim.pb, sim.prec, sim.basis, ev, b["tape"], b["B"])
    nv.mts_backward(sim.pb, sim.prec, sim.basis, ev, b["tape"], None, b["gl"], b["g"])


@pytest.mark.parametrize("case", ["8x8", "ragged128"])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_step_replays_in_a_graph(case, prec):
    from paper_2503_18479_gb300 import native as nv
    from paper_2503_18479_gb300.simulator import Simulator
    wl = small_8x8(n_cfg=300) if case == "8x8" else \
        small_ragged(n_struct=5, seed=11, grid=8, max_freq=2, ports=(1, 16, 64, 128))
    sim = Simulator(wl, prec)
    n = wl.n_cfg
    rng = np.random.Generator(np.random.PCG64(21))
    Cg = torch.from_numpy(wl.C).cuda()
    evg = sim.make_eval(Cg, True)
    bg = _buffers(sim, n)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        _step(nv, sim, evg, bg)  # eager warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        _step(nv, sim, evg, bg)
    for rep in range(2):
        Cnew = torch.from_numpy(rng.uniform(20e-12, 200e-12, wl.C.shape)).cuda()
        Cg.copy_(Cnew)
        graph.replay()
        be = _buffers(sim, n)
        _step(nv, sim, sim.make_eval(Cnew, True), be)
        torch.cuda.synchronize()
        for k in ("B", "loss", "g"):
            assert torch.equal(bg[k], be[k]), (rep, k)
        assert sim.status(bg["tape"], n) == (0, 0)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_sroute_step_replays_in_a_graph(prec):
    """The S-parameter route's step (series-RC loads, forward with the field and objective,
    adjoint, dL/dC) captured once and replayed on new capacitances equals eager calls."""
    from paper_2503_18479_gb300 import native as nv
    from paper_2503_18479_gb300 import workloads as W
    from paper_2503_18479_gb300.sroute import SRoute
    wl = W.sroute_array(3, 2, seed=4, n_cfg=40, grid=10)
    sr = SRoute(wl.S0, wl.field, wl.rows, wl.cols, wl.n1, sc_const=wl.sc_const,
                loss_idx=wl.loss_idx, target=wl.target, precision=prec)
    n, F, nS = wl.n_cfg, sr.F, sr.nS
    R = torch.from_numpy(wl.R).cuda()
    om = torch.from_numpy(wl.omega).cuda()

    def bufs():
        return dict(svar=torch.empty((n, F, nS, 2), dtype=torch.float64, device="cuda"),
                    tape=sr.alloc_tape(n),
                    B=torch.empty((n, sr.n1, F, sr.P), dtype=sr.b_dtype, device="cuda"),
                    loss=torch.empty(n, dtype=torch.float64, device="cuda"),
                    gs=torch.empty((n, F, nS, 2), dtype=torch.float64, device="cuda"),
                    gC=torch.empty((n, nS), dtype=torch.float64, device="cuda"))

    gl = torch.ones(n, dtype=torch.float64, device="cuda")

    def step(C, b):
        ev = nv.SrouteEval(b["svar"], sr.target, sr.loss_mode)
        nv.mts_rc_reflection(n, F, nS, om, R, C, wl.Z0, nS, 0, b["svar"])
        nv.mts_sroute_forward(sr.sp, sr.prec, sr.sbasis, ev, B_out=b["B"], loss_out=b["loss"],
                              tape=b["tape"])
        nv.mts_sroute_backward(sr.sp, sr.prec, sr.sbasis, ev, b["tape"], grad_loss=gl,
                               grad_svar=b["gs"])
        nv.mts_rc_reflection_vjp(n, F, nS, om, R, C, wl.Z0, nS, 0, b["gs"], grad_C=b["gC"])

    Cg = torch.from_numpy(wl.C).cuda()
    bg = bufs()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step(Cg, bg)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step(Cg, bg)
    rng = np.random.Generator(np.random.PCG64(22))
    for rep in range(2):
        Cnew = torch.from_numpy(rng.uniform(20e-12, 200e-12, wl.C.shape)).cuda()
        Cg.copy_(Cnew)
        graph.replay()
        be = bufs()
        step(Cnew, be)
        torch.cuda.synchronize()
        for k in ("B", "loss", "gC"):
            assert torch.equal(bg[k], be[k]), (rep, k)
