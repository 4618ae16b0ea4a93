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
# (|b| carries ~1e-7, amplified by |b| / ||b| - t| near a target), and a structure's sum over
# frequencies of Re or Im(mu_k I_k) can cancel: on a one-port structure whose dloss/dL is
# 1e-3 of its per-frequency terms the relative error reached 7e-5 (measured). Bounds: the
# whole tensor within 1e-6 with cosine >= 0.9999 (the spec measure, as for dloss/dC);
# per structure within 1e-5 relative or 1e-6 of the whole tensor's norm; MTS_FP64 every
# structure within 1e-10.
TOL = {"fp64": 1e-10, "mixed": 1e-5}
TOL_ALL = {"fp64": 1e-10, "mixed": 1e-6}


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
    gR, gL = gR.cpu().numpy(), gL.cpu().numpy()
    allR = np.concatenate([gl[:, s:s + 1] * refs[s][0] for s in range(len(wl.structures))], axis=1)
    allL = np.concatenate([gl[:, s:s + 1] * refs[s][1] for s in range(len(wl.structures))], axis=1)
    assert rel(gR, allR) < TOL_ALL[prec] and rel(gL, allL) < TOL_ALL[prec]
    assert cosine(gR, allR) >= 0.9999 and cosine(gL, allL) >= 0.9999
    nR, nL = np.linalg.norm(allR), np.linalg.norm(allL)
    gR, gL = split_ports(wl, gR), split_ports(wl, gL)
    for s in range(len(wl.structures)):
        wantR = gl[:, s:s + 1] * refs[s][0]
        wantL = gl[:, s:s + 1] * refs[s][1]
        for got, want, nrm in ((gR[s], wantR, nR), (gL[s], wantL, nL)):
            err = np.linalg.norm(got - want)
            if prec == "fp64":
                assert err <= TOL[prec] * np.linalg.norm(want), (s, rel(got, want))
            else:
                assert err <= max(TOL[prec] * np.linalg.norm(want), TOL_ALL[prec] * nrm), \
                    (s, rel(got, want))


@pytest.mark.parametrize("name", ["8x8", "ragged128"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_omega_and_drive_gradients_match_oracle(name, prec):
    """dloss/domega (drive fixed) and the drive cotangent conj(mu) per structure against the
    oracle's adjoint forms (pinned by central differences)."""
    from paper_2503_18479_gb300.simulator import Simulator
    wl, _ = _case(name)
    sim = Simulator(wl, prec)
    out = sim.forward(torch.from_numpy(wl.C).cuda(), want_B=False)
    gR, gL, gw, gV = sim.param_grad(out["ev"], out["tape"], with_omega=True)
    gw, gV = gw.cpu().numpy(), gV.cpu().numpy()
    fo = np.concatenate([[0], np.cumsum([st.n_freq for st in wl.structures])])
    vo = np.concatenate([[0], np.cumsum([st.n_freq * st.n_ports for st in wl.structures])])
    want_w, want_V = [], []
    for s, st in enumerate(wl.structures):
        H, M = structure_basis(wl, s)
        w_s, V_s = oracle.gradient_omega_v(H, M, st.R, wl.structure_C(s), st.omega, st.V,
                                           st.loss_idx, wl.structure_target(s))
        want_w.append(w_s)
        want_V.append(V_s.reshape(wl.n_cfg, -1))
        got_w, got_V = gw[:, fo[s]:fo[s + 1]], gV[:, vo[s]:vo[s + 1]]
        if prec == "fp64":
            assert rel(got_w, w_s) < 1e-10, (s, rel(got_w, w_s))
            assert rel(got_V, V_s.reshape(wl.n_cfg, -1)) < 1e-10
    if prec == "mixed":  # whole-tensor bounds (per-structure sums can cancel, as for dR/dL)
        assert rel(gw, np.concatenate(want_w, axis=1)) < 1e-6
        assert rel(gV, np.concatenate(want_V, axis=1)) < 1e-6
        assert cosine(gw, np.concatenate(want_w, axis=1)) >= 0.9999
