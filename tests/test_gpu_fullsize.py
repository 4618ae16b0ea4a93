"""Parity at the benchmark's full sizes, in the launch configuration bench.py times (one
batch, the library's default schedule): the CUDA path runs every configuration; the FP64
oracle recomputes a sample of configurations (all their points, or a sample of points for
the largest array) and their objective and dloss/dC. Tolerances as in test_gpu_parity
(MTS_MIXED: 1e-6 on B, the loss and the gradient; 5e-6 on B of the K = 1024 tensor path). A
sampled configuration can sit close to its target, where the objective is a small difference
of nearly equal fields: its error is then measured against the objective's sensitivity to the
field (helpers.loss_err), not against the objective alone."""
import numpy as np
import pytest
import torch

import oracle
from helpers import apply_target_rule, loss_err, rel, structure_basis
from paper_2503_18479_gb300 import build_lib
from paper_2503_18479_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    build_lib.build()


def _gpu_step(wl, prec="mixed"):
    """The bench step: solve + objective + adjoint, superposition, gradient combine."""
    from paper_2503_18479_gb300 import native as nv
    from paper_2503_18479_gb300.simulator import Simulator
    sim = Simulator(wl, prec)
    n = wl.n_cfg
    C = torch.from_numpy(wl.C).cuda()
    ev = sim.make_eval(C, True)
    tape = sim.alloc_tape(n)
    B = torch.empty((n, sim.sumFP), dtype=sim.b_dtype, device="cuda")
    loss = torch.empty((n, sim.n_struct), dtype=torch.float64, device="cuda")
    g = torch.empty((n, sim.n_ports), dtype=torch.float64, device="cuda")
    ones = torch.ones((n, sim.n_struct), dtype=torch.float64, device="cuda")
    nv.mts_solve(sim.pb, sim.prec, sim.basis, ev, None, loss, tape)
    nv.mts_superpose(sim.pb, sim.prec, sim.basis, ev, tape, B)
    nv.mts_backward(sim.pb, sim.prec, sim.basis, ev, tape, None, ones, g)
    torch.cuda.synchronize()
    assert sim.status(tape, n) == (0, 0)
    return sim, B, loss, g


def _check_single(wl, n_sample, seed, tol_b=1e-6):
    st = wl.structures[0]
    sim, B, loss, g = _gpu_step(wl)
    rng = np.random.Generator(np.random.PCG64(seed))
    cfg = np.sort(rng.choice(wl.n_cfg, size=min(n_sample, wl.n_cfg), replace=False))
    H, M = structure_basis(wl, 0)
    t = wl.structure_target(0)
    ref = oracle.forward(H, M, st.R, wl.C[cfg], st.omega, st.V, st.loss_idx, t)
    gref = oracle.gradient(H, M, st.R, wl.C[cfg], st.omega, st.V, st.loss_idx, t)
    idx = torch.from_numpy(cfg).cuda()
    Bg = B[idx].cpu().numpy().reshape(ref["B"].shape)
    assert rel(Bg, ref["B"]) < tol_b, rel(Bg, ref["B"])
    err = loss_err(loss[idx, 0].cpu().numpy(), ref, st.loss_idx)
    assert err < 1e-6, err
    assert rel(g[idx].cpu().numpy(), gref) < 1e-6


def test_array_8x8_full():
    """4096 configurations x 65,600 points at 63.6 MHz; 64 configurations checked in full."""
    _check_single(W.array_8x8(seed=0), 64, seed=1)


def test_line_8x1_full():
    """1024 configurations x 201 frequencies x 4104 points; 24 configurations checked."""
    _check_single(apply_target_rule(W.line_8x1(seed=0)), 24, seed=2)


def test_single_loop_full():
    """The single loop: 1 configuration x 101 frequencies, checked in full."""
    _check_single(apply_target_rule(W.single_loop(seed=0)), 1, seed=3)


def test_ragged_full():
    """10,000 structures of 1..128 ports in one batch; 40 structures checked in full."""
    wl = W.ragged(seed=0)
    sim, B, loss, g = _gpu_step(wl)
    rng = np.random.Generator(np.random.PCG64(4))
    fo = np.concatenate([[0], np.cumsum([s.n_freq * s.n_points for s in wl.structures])])
    po = wl.port_off()
    Bh, lh, gh = B[0].cpu().numpy(), loss[0].cpu().numpy(), g[0].cpu().numpy()
    for s in np.sort(rng.choice(len(wl.structures), size=40, replace=False)):
        st = wl.structures[s]
        H, M = structure_basis(wl, s)
        t = wl.structure_target(s)
        C = wl.structure_C(s)
        ref = oracle.forward(H, M, st.R, C, st.omega, st.V, st.loss_idx, t)
        gref = oracle.gradient(H, M, st.R, C, st.omega, st.V, st.loss_idx, t)
        assert rel(Bh[fo[s]:fo[s + 1]], ref["B"][0].ravel()) < 1e-6, s
        assert rel(lh[s], ref["loss"][0]) < 1e-6, s
        assert rel(gh[po[s]:po[s + 1]], gref[0]) < 1e-6, s


def test_array_32x32_full():
    """1024 ports, 65,536 segments, 256 configurations x 1,048,576 + 1024 points; 3
    configurations checked (objective, gradient, and 4096 sampled points of B)."""
    wl = W.array_32x32(seed=0)
    st = wl.structures[0]
    sim, B, loss, g = _gpu_step(wl)
    rng = np.random.Generator(np.random.PCG64(5))
    cfg = np.sort(rng.choice(wl.n_cfg, size=3, replace=False))
    pts = np.sort(rng.choice(st.n_points, size=4096, replace=False))
    Hs = oracle.basis(st.loop_vtx_off, st.vx, st.vy, st.vz, st.px[pts], st.py[pts], st.pz[pts],
                      wl.wire_radius)
    HL = oracle.basis(st.loop_vtx_off, st.vx, st.vy, st.vz, st.px[st.loss_idx],
                      st.py[st.loss_idx], st.pz[st.loss_idx], wl.wire_radius)
    status, M = oracle.inductance(st.loop_vtx_off, st.vx, st.vy, st.vz, wl.wire_radius, st.L_self)
    assert status == 0
    t = wl.structure_target(0)
    li = np.arange(len(st.loss_idx))
    ref = oracle.forward(HL, M, st.R, wl.C[cfg], st.omega, st.V, li, t, want_B=False)
    gref = oracle.gradient(HL, M, st.R, wl.C[cfg], st.omega, st.V, li, t)
    Iref = ref["I"][:, 0, :]
    idx = torch.from_numpy(cfg).cuda()
    Bg = B[idx][:, torch.from_numpy(pts).cuda()].cpu().numpy()
    assert rel(Bg, Iref @ Hs.T) < 5e-6, rel(Bg, Iref @ Hs.T)
    assert rel(loss[idx, 0].cpu().numpy(), ref["loss"]) < 1e-6
    assert rel(g[idx].cpu().numpy(), gref) < 1e-6


def test_sroute_array_full():
    """The scattering-parameter route on the 8x8-plus-drive workload at the bench's size
    (4096 configurations, 65,600 points, 65 structure ports, MTS_MIXED): 8 configurations
    checked in full (Bcomb, objective, dL/dC through Eq. 3)."""
    from paper_2503_18479_gb300.sroute import SRoute, rc_reflection
    wl = W.sroute_array(seed=0)
    sr = SRoute(wl.S0, wl.field, wl.rows, wl.cols, wl.n1, sc_const=wl.sc_const,
                loss_idx=wl.loss_idx, target=wl.target, precision="mixed")
    C = torch.from_numpy(wl.C).cuda().requires_grad_(True)
    gam = rc_reflection(torch.from_numpy(wl.R).cuda(), C, torch.from_numpy(wl.omega).cuda(), wl.Z0)
    B, loss = sr(gam)
    loss.sum().backward()
    torch.cuda.synchronize()
    rng = np.random.Generator(np.random.PCG64(6))
    cfg = np.sort(rng.choice(wl.n_cfg, size=8, replace=False))
    w = wl.omega[None, :, None]
    Zl = wl.R[cfg][:, None, :] - 1j / (w * wl.C[cfg][:, None, :])
    svar = (Zl - wl.Z0) / (Zl + wl.Z0)  # Eq. 3
    ref = oracle.sroute_pipeline(wl.S0, wl.field, wl.sc_const, wl.rows, wl.cols, svar,
                                 wl.loss_idx, wl.target)
    idx = torch.from_numpy(cfg).cuda()
    assert rel(B.detach()[idx].cpu().numpy(), ref["B"]) < 1e-6
    assert rel(loss.detach()[idx].cpu().numpy(), ref["loss"]) < 1e-6
    g = oracle.sroute_gradient(wl.S0, wl.field, wl.sc_const, wl.rows, wl.cols, svar,
                               wl.loss_idx, wl.target)
    dgam = 2 * wl.Z0 / (Zl + wl.Z0) ** 2 * (1j / (w * wl.C[cfg][:, None, :] ** 2))
    gC = np.real(np.conj(g) * dgam).sum(axis=1)
    assert rel(C.grad[idx].cpu().numpy(), gC) < 1e-6
