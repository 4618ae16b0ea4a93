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


def test_static_solve_reports_unconverged_systems():
    """A system too ill-conditioned for FP32 factors (an eigenvalue of A of about R = 1e-9
    ohm, condition number about 3e10) cannot meet the refinement tolerance: after
    mts_solve_static, mts_solve_static_status reports MTS_ENOCONV with exactly that system
    counted, and a well-conditioned batch reports MTS_OK. The static path's status words are
    the ones mts_solve would have written to a tape."""
    import dataclasses
    assert torch.cuda.is_available()
    build_lib.build()
    from helpers import small_rect, structure_basis
    from paper_2503_18479_gb300 import native as nv
    from paper_2503_18479_gb300.simulator import Simulator
    wl = small_rect(8, 8, n_cfg=6)
    st = dataclasses.replace(wl.structures[0], R=np.full(wl.structures[0].n_ports, 1e-9))
    wl = dataclasses.replace(wl, structures=[st])
    _, M = structure_basis(wl, 0)  # the oracle's inductances choose the planted input
    w0 = float(st.omega[0])
    C0 = 1.0 / (w0 * w0 * float(np.linalg.eigvalsh(M)[0]))
    sim = Simulator(wl, "mixed")
    n = wl.n_cfg
    C = torch.from_numpy(wl.C).cuda()
    nv.mts_solve_static(sim.pb, sim.prec, sim.basis, sim.make_eval(C, True))
    assert nv.mts_solve_static_status(sim.pb, n, sim.prec) == (nv.MTS_OK, 0)
    Cbad = C.clone()
    Cbad[2, :] = C0
    I = torch.empty((n, sim.sumFN), dtype=torch.complex128, device="cuda")
    nv.mts_solve_static(sim.pb, sim.prec, sim.basis, sim.make_eval(Cbad, True), I)
    code, n_bad = nv.mts_solve_static_status(sim.pb, n, sim.prec)
    assert code == nv.MTS_ENOCONV and n_bad == 1, (code, n_bad)
    assert torch.isfinite(torch.view_as_real(I)).all()  # results are written either way
