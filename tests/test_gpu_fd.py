"""The adjoint gradient of the CUDA path against central finite differences of the CUDA
path's own objective (MTS_FP64, so that the difference quotient is not lost in rounding),
h = 1e-3 pF as the paper-shaped workloads prescribe, on 16 capacitors; and systems with a
non-finite capacitance, or too ill-conditioned for FP32 factors to converge, are flagged
without disturbing the others."""
import numpy as np
import pytest
import torch

from helpers import small_8x8, small_rect, structure_basis
from paper_2503_18479_gb300 import build_lib
from paper_2503_18479_gb300 import workloads as W

pytestmark = pytest.mark.gpu

H_FD = 1e-15  # 1e-3 pF


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    build_lib.build()


def _loss(sim, C):
    return sim.forward(C, want_B=False)["loss"]


@pytest.mark.parametrize("case", ["8x8", "10x8", "32x32"])
def test_adjoint_matches_central_differences(case):
    from paper_2503_18479_gb300.simulator import Simulator
    if case == "8x8":
        wl = small_8x8(n_cfg=2, grid=8, planes=(0.02,))
    elif case == "10x8":
        wl = small_rect(10, 8, n_cfg=2, n_freq=2, grid=8, seed=6)
    else:
        wl = W.array_32x32(seed=5, n_cfg=2, grid=8, planes=(0.02,), seg_per_side=2)
    sim = Simulator(wl, "fp64")
    C0 = torch.from_numpy(wl.C).cuda().requires_grad_(True)
    _, loss = sim(C0, want_B=False)
    loss.sum().backward()
    g = C0.grad.cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(12))
    ks = rng.choice(wl.n_ports, size=16, replace=False)
    fd = np.zeros((wl.n_cfg, 16))
    for i, k in enumerate(ks):
        Cp = torch.from_numpy(wl.C.copy()).cuda()
        Cm = Cp.clone()
        Cp[:, k] += H_FD
        Cm[:, k] -= H_FD
        fd[:, i] = ((_loss(sim, Cp) - _loss(sim, Cm)) / (2 * H_FD)).cpu().numpy()[:, 0]
    ga = g[:, ks]
    err = np.linalg.norm(ga - fd) / np.linalg.norm(fd)
    assert err < 1e-5, err  # O(h^2) truncation plus FP64 rounding of the difference
    cos = float((ga * fd).sum() / (np.linalg.norm(ga) * np.linalg.norm(fd)))
    assert cos >= 0.9999


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_non_finite_capacitance_is_flagged(prec):
    from paper_2503_18479_gb300.simulator import Simulator
    wl = small_8x8(n_cfg=8, grid=8, planes=(0.02,))
    sim = Simulator(wl, prec)
    C = torch.from_numpy(wl.C).cuda()
    ref = sim.forward(C)
    Cbad = C.clone()
    Cbad[3, 5] = float("nan")
    out = sim.forward(Cbad)
    torch.cuda.synchronize()
    code, n_bad = sim.status(out["tape"], wl.n_cfg)
    assert n_bad == 1 and code != 0
    # which system: mts_system_status copies the per-system words
    from paper_2503_18479_gb300 import native as nv
    words = torch.full((wl.n_cfg, sim.omega.numel()), -1, dtype=torch.int32, device="cuda")
    nv.mts_system_status(sim.pb, wl.n_cfg, sim.prec, out["tape"], words)
    w = words.cpu().numpy()
    assert w[3, 0] == 2 and np.count_nonzero(w) == 1, w
    keep = [b for b in range(8) if b != 3]
    assert torch.equal(out["B"][keep], ref["B"][keep])
    assert torch.equal(out["loss"][keep], ref["loss"][keep])


@pytest.mark.parametrize("prec", ["mixed", "bf16"])
@pytest.mark.parametrize("shape", [(4, 4), (8, 8), (9, 8)])
def test_unconverged_system_is_flagged(prec, shape):
    """A configuration tuned so that A = R + jwM + 1/(jwC) has an eigenvalue of about R =
    1e-9 ohm (every C at 1/(w^2 mu), mu the smallest eigenvalue of M; condition number about
    3e10) cannot be solved from FP32 factors: rounding A to FP32 moves that eigenvalue by
    about 1e-6 ohm, so each refinement correction is as large as the last and the system
    must report status 1 (missed the tolerance) at that frequency only. Covers the
    register kernels for 16 and 64 ports and the blocked kernel for 72; the other systems
    (condition numbers below 1e3) keep status 0 and bit-identical results."""
    import dataclasses
    from paper_2503_18479_gb300 import native as nv
    from paper_2503_18479_gb300.simulator import Simulator
    nx, ny = shape
    wl = small_rect(nx, ny, n_cfg=6)
    st = dataclasses.replace(wl.structures[0], R=np.full(wl.structures[0].n_ports, 1e-9))
    wl = dataclasses.replace(wl, structures=[st])
    _, M = structure_basis(wl, 0)  # the oracle's inductances choose the planted input
    w0 = float(st.omega[0])
    C0 = 1.0 / (w0 * w0 * float(np.linalg.eigvalsh(M)[0]))
    sim = Simulator(wl, prec)
    C = torch.from_numpy(wl.C).cuda()
    ref = sim.forward(C)
    bad_cfg = 2
    Cbad = C.clone()
    Cbad[bad_cfg, :] = C0
    out = sim.forward(Cbad)
    code, n_bad = sim.status(out["tape"], wl.n_cfg)
    assert code == nv.MTS_ENOCONV and n_bad == 1, (code, n_bad)
    words = torch.full((wl.n_cfg, sim.omega.numel()), -1, dtype=torch.int32, device="cuda")
    nv.mts_system_status(sim.pb, wl.n_cfg, sim.prec, out["tape"], words)
    w = words.cpu().numpy()
    want = np.zeros_like(w)
    want[bad_cfg, 0] = 1
    assert np.array_equal(w, want), w
    code_ref, n_ref = sim.status(ref["tape"], wl.n_cfg)
    assert code_ref == nv.MTS_OK and n_ref == 0
    keep = [b for b in range(wl.n_cfg) if b != bad_cfg]
    assert torch.equal(out["B"][keep], ref["B"][keep])
    assert torch.equal(out["loss"][keep], ref["loss"][keep])
    assert torch.isfinite(out["B"][bad_cfg]).all()  # results are written either way
