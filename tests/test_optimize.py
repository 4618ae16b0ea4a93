"""The optimisation loop (paper Sec. III-C: Adam, learning rate 1e-13; Sec. V-B: clipping or
tanh projection): the Adam step against torch.optim.Adam, the projections, graph replay
against eager epochs, and a whole fit against the same Adam driven by the FP64 oracle's
objective and gradient on the CPU."""
import numpy as np
import pytest
import torch

import oracle
from helpers import small_loop, structure_basis
from paper_2503_18479_gb300 import build_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    build_lib.build()


def _adam_ref(theta, grads, lr, betas, eps):
    p = torch.nn.Parameter(theta.clone())
    opt = torch.optim.Adam([p], lr=lr, betas=betas, eps=eps)
    for g in grads:
        opt.zero_grad()
        p.grad = g.clone()
        opt.step()
    return p.detach()


def test_adam_step_matches_torch_adam():
    from paper_2503_18479_gb300 import native as nv
    rng = np.random.Generator(np.random.PCG64(3))
    n, steps = 1000, 5
    theta = torch.from_numpy(rng.uniform(20e-12, 200e-12, n))
    grads = [torch.from_numpy(rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3)) for _ in range(steps)]
    want = _adam_ref(theta, grads, 1e-13, (0.9, 0.999), 1e-8)
    C = theta.cuda().clone()
    m = torch.zeros(n, dtype=torch.float64, device="cuda")
    v = torch.zeros_like(m)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    opt = nv.MtsAdam(1e-13, 0.9, 0.999, 1e-8, nv.MTS_PROJ_NONE, 0.0, 0.0)
    for g in grads:
        nv.mts_adam_step(n, opt, C, None, g.cuda(), m, v, step)
    torch.cuda.synchronize()
    assert int(step.item()) == steps
    rel = float((C.cpu() - want).abs().max() / want.abs().max())
    assert rel < 1e-14, rel


def test_projections():
    from paper_2503_18479_gb300 import native as nv
    n = 257
    g = torch.linspace(-1.0, 1.0, n, dtype=torch.float64, device="cuda") * 1e3
    lo, hi = 20e-12, 200e-12
    # clipping: large steps push values outside; they end on the bounds
    C = torch.full((n,), 110e-12, dtype=torch.float64, device="cuda")
    m, v = torch.zeros_like(C), torch.zeros_like(C)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    opt = nv.MtsAdam(1e-9, 0.9, 0.999, 1e-8, nv.MTS_PROJ_CLIP, lo, hi)
    nv.mts_adam_step(n, opt, C, None, g, m, v, step)
    torch.cuda.synchronize()
    assert float(C.min()) == lo and float(C.max()) == hi
    # tanh: C follows u through c_mid + c_half tanh(u), strictly inside the range
    u = torch.linspace(-2.0, 2.0, n, dtype=torch.float64, device="cuda")
    C = 110e-12 + 90e-12 * torch.tanh(u)
    m, v = torch.zeros_like(C), torch.zeros_like(C)
    step.zero_()
    opt = nv.MtsAdam(1e-2, 0.9, 0.999, 1e-30, nv.MTS_PROJ_TANH, lo, hi)
    u0 = u.clone()
    nv.mts_adam_step(n, opt, C, u, g, m, v, step)
    torch.cuda.synchronize()
    assert torch.allclose(C, 110e-12 + 90e-12 * torch.tanh(u), rtol=1e-15, atol=0)
    assert bool(((C > lo) & (C < hi)).all())
    # chain rule through the projection: the first Adam step moves u by -lr sign(g_u)
    gu = g * 90e-12 * (1 - torch.tanh(u0) ** 2)
    assert torch.allclose(u0 - u, 1e-2 * torch.sign(gu), rtol=1e-6, atol=1e-12)


def test_graph_replay_equals_eager_epochs():
    from paper_2503_18479_gb300.optimize import AdamFit
    from paper_2503_18479_gb300.simulator import Simulator
    wl = small_loop(n_cfg=6, n_freq=5, grid=8)
    sim = Simulator(wl, "fp64")
    C0 = torch.from_numpy(wl.C)
    a = AdamFit(sim, C0, max_epochs=30, use_graph=True)
    b = AdamFit(sim, C0, max_epochs=30, use_graph=False)
    Ca, ha = a.run(30)
    Cb, hb = b.run(30)
    assert torch.equal(Ca, Cb)
    assert torch.equal(ha, hb)


def test_fit_matches_oracle_driven_adam():
    """40 epochs at the paper's learning rate on four single-loop fits: GPU (MTS_FP64, CUDA
    graph) against torch.optim.Adam fed by the oracle's objective and gradient."""
    from paper_2503_18479_gb300.optimize import AdamFit
    from paper_2503_18479_gb300.simulator import Simulator
    wl = small_loop(n_cfg=4, n_freq=5, grid=8)
    st = wl.structures[0]
    H, M = structure_basis(wl, 0)
    t = wl.structure_target(0)
    sim = Simulator(wl, "fp64")
    epochs = 40
    fit = AdamFit(sim, torch.from_numpy(wl.C), lr=1e-13, max_epochs=epochs)
    C_gpu, hist = fit.run(epochs)
    p = torch.nn.Parameter(torch.from_numpy(wl.C.copy()))
    opt = torch.optim.Adam([p], lr=1e-13)
    losses = []
    for _ in range(epochs):
        Cn = p.detach().numpy()
        out = oracle.forward(H, M, st.R, Cn, st.omega, st.V, st.loss_idx, t, want_B=False)
        losses.append(out["loss"])
        g = oracle.gradient(H, M, st.R, Cn, st.omega, st.V, st.loss_idx, t)
        opt.zero_grad()
        p.grad = torch.from_numpy(g)
        opt.step()
    C_ref = p.detach().numpy()
    C_g = C_gpu.cpu().numpy()
    assert np.max(np.abs(C_g - C_ref)) / np.max(np.abs(C_ref)) < 1e-9
    h = hist.cpu().numpy()[:, :, 0]
    L = np.array(losses)
    assert np.max(np.abs(h - L)) / np.max(np.abs(L)) < 1e-9
    assert (L[-1] < L[0]).all()  # every fit improved
