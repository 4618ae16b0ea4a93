"""dloss/dR and dloss/dL (self inductances) of the CUDA path (mts_param_grad, after a forward
with the objective) against the FP64 oracle's adjoint form (itself pinned by central
differences), for one structure, a ragged batch with 128-port structures, and a
per-structure loss cotangent."""
import numpy as np
import pytest
import torch

import oracle
from helpers import cosine, rel, small_8x8, small_ragged, small_rect, split_ports, structure_basis
from paper_2503_18479_gb300 import build_lib

pytestmark = pytest.mark.gpu

# MTS_MIXED evaluates the objective's cotangent G = 2 (|b| - t) b/|b| from an FP32 basis
# (|b| carries ~1e-7), which |b| / ||b| - t| amplifies where the field is near its target;
# -Re(mu_k I_k) can cancel further. Per structure, down to a single port, that reaches
# 1.0e-6 (measured), so the bound for these extra outputs is 2e-6.
TOL = {"fp64": 1e-10, "mixed": 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    build_lib.build()


_CASES = {
    "8x8": lambda: small_8x8(n_cfg=50, grid=12, planes=(0.02,)),
    "ragged128": lambda: small_ragged(n_struct=5, seed=8, grid=8, max_freq=6, ports=(1, 8, 64, 128)),
    "10x8": lambda: small_rect(10, 8, n_cfg=8, n_freq=2, grid=8, seed=2),
}
_cache = {}


def _case(name):
    if name not in _cache:
        wl = _CASES[name]()
        refs = []
        for s, st in enumerate(wl.structures):
            H, M = structure_basis(wl, s)
            refs.append(oracle.gradient_rl(H, M, st.R, wl.structure_C(s), st.omega, st.V,
                                           st.loss_idx, wl.structure_target(s)))
        _cache[name] = (wl, refs)
    return _cache[name]


@pytest.mark.parametrize("name", list(_CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_param_grad_matches_oracle(name, prec):
    from paper_2503_18479_gb300.simulator import Simulator
    wl, refs = _case(name)
    sim = Simulator(wl, prec)
    out = sim.forward(torch.from_numpy(wl.C).cuda(), want_B=False)
    rng = np.random.Generator(np.random.PCG64(4))
    gl = rng.uniform(0.5, 2.0, (wl.n_cfg, len(wl.structures)))
    gR, gL = sim.param_grad(out["ev"], out["tape"], torch.from_numpy(gl).cuda())
    gR, gL = split_ports(wl, gR.cpu().numpy()), split_ports(wl, gL.cpu().numpy())
    for s in range(len(wl.structures)):
        wantR = gl[:, s:s + 1] * refs[s][0]
        wantL = gl[:, s:s + 1] * refs[s][1]
        assert rel(gR[s], wantR) < TOL[prec], (s, rel(gR[s], wantR))
        assert rel(gL[s], wantL) < TOL[prec], (s, rel(gL[s], wantL))
        assert cosine(gR[s], wantR) >= 0.9999 and cosine(gL[s], wantL) >= 0.9999
