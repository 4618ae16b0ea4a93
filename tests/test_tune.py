"""Schedules and the autotuner: every superposition schedule (all structures on the tensor
cores, the default threshold, all on the SIMT kernel), every CTA size of the blocked solve and
every width of the register classes give the oracle's results; the autotuner returns one of
its candidates and the tuned Simulator still matches."""
import numpy as np
import pytest
import torch

from helpers import oracle_reference, rel, small_ragged, small_rect, split_B, structure_basis
from paper_2503_18479_gb300 import build_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    build_lib.build()


_wl = {}


def _ragged():
    if "r" not in _wl:
        wl = small_ragged(n_struct=6, seed=8, grid=8, max_freq=24, ports=(1, 8, 64, 128))
        _wl["r"] = (wl, oracle_reference(wl, bases=[structure_basis(wl, s)
                                                    for s in range(len(wl.structures))]))
    return _wl["r"]


@pytest.mark.parametrize("simt_max_sys", [-1, 0, 1 << 30])
@pytest.mark.parametrize("prec", ["mixed", "bf16"])
def test_superposition_schedules_agree(simt_max_sys, prec):
    from paper_2503_18479_gb300.simulator import Simulator
    wl, ref = _ragged()
    sim = Simulator(wl, prec)
    sim.tuning = {"simt_max_sys": simt_max_sys, "large_threads": 0}
    out = sim.forward(torch.from_numpy(wl.C).cuda())
    Bs = split_B(wl, out["B"].cpu().numpy())
    tol = 1e-6 if prec == "mixed" else 1e-2
    for s in range(len(wl.structures)):
        assert rel(Bs[s], ref[s]["B"]) < tol, (s, rel(Bs[s], ref[s]["B"]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_large_solve_cta_sizes_agree(prec):
    """The blocked solve of 80-port systems with 128, 256 and 512 threads: with MTS_MIXED the
    first keeps the matrix in the factor scratch and the others in shared memory (a backward
    with a field cotangent reloads the forward's factors into it); the same results to
    rounding, for the loss cotangent alone and with a field cotangent."""
    from paper_2503_18479_gb300.simulator import Simulator
    wl = small_rect(10, 8, n_cfg=6, n_freq=2, grid=8, seed=9)
    sim = Simulator(wl, prec)
    outs = []
    gB = None
    for lt in (128, 256, 512):
        sim.tuning = {"simt_max_sys": 0, "large_threads": lt}
        C = torch.from_numpy(wl.C).cuda().requires_grad_(True)
        B, loss = sim(C)
        loss.sum().backward()
        C2 = torch.from_numpy(wl.C).cuda().requires_grad_(True)
        B2, loss2 = sim(C2)
        if gB is None:
            g = torch.Generator().manual_seed(3)
            gB = torch.complex(torch.randn(B2.shape, generator=g, dtype=torch.float64),
                               torch.randn(B2.shape, generator=g, dtype=torch.float64))
            gB = gB.to(B2.dtype).cuda()
        torch.autograd.backward([B2, loss2], [gB, torch.ones_like(loss2)])
        outs.append((B.detach(), loss.detach(), C.grad.clone(), C2.grad.clone()))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_register_class_widths_agree(prec):
    """The register classes of up to 32 ports in their own mapping or one wider (reg_widen):
    the same results to rounding, and the oracle's."""
    from paper_2503_18479_gb300.simulator import Simulator
    wl = small_ragged(n_struct=6, seed=5, grid=8, max_freq=6, ports=(1, 8, 16, 32))
    ref = oracle_reference(wl, bases=[structure_basis(wl, s) for s in range(len(wl.structures))])
    sim = Simulator(wl, prec)
    outs = []
    for w in (0, 1, 2, 4, 7):
        sim.tuning = {"simt_max_sys": 0, "large_threads": 0, "reg_widen": w}
        C = torch.from_numpy(wl.C).cuda().requires_grad_(True)
        B, loss = sim(C)
        loss.sum().backward()
        outs.append((B.detach().cpu().numpy(), loss.detach().cpu().numpy(), C.grad.cpu().numpy()))
    # different widths block the LU differently: FP32 factors round differently and the
    # refinement converges to its tolerance (1e-8 estimated), not to the same bits
    tol = 1e-13 if prec == "fp64" else 1e-7
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert rel(a, b) < tol
    Bs = split_B(wl, outs[-1][0])
    for s in range(len(wl.structures)):
        assert rel(Bs[s], ref[s]["B"]) < (1e-10 if prec == "fp64" else 1e-6)


def test_autotune_picks_a_candidate_and_keeps_results():
    from paper_2503_18479_gb300 import tune
    from paper_2503_18479_gb300.simulator import Simulator
    wl, ref = _ragged()
    sim = Simulator(wl, "mixed")
    C = torch.from_numpy(wl.C).cuda()
    tuning, times = tune.autotune(sim, C, reps=2)
    assert (tuning["simt_max_sys"], tuning["large_threads"], tuning["reg_widen"]) in times
    assert len(times) >= len(tune.SIMT_CHOICES) * len(tune.LARGE_CHOICES)
    assert all(np.isfinite(t) and t > 0 for t in times.values())
    out = sim.forward(C)
    Bs = split_B(wl, out["B"].cpu().numpy())
    for s in range(len(wl.structures)):
        assert rel(Bs[s], ref[s]["B"]) < 1e-6
